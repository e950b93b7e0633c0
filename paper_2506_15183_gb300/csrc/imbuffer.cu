// Second-eye synthesis through a row-downsampled intermediate buffer (ImBuffer):
// strategies (c) "resolution-independent intermediate buffers" and (d) "linear
// interpolation" of the Reprojector.
//
// The paper states their intent only; the reading implemented here (and in the
// oracle, step for step):
//   s in {1, 2, 4, 8, 16} cells per row pixel group; row y has ws = ceil(w / s) cells,
//   cell i standing for source pixels s i .. s i + s - 1.
//   1. Alg. 1 per cell on its representative pixel p = min(s i + s/2, w - 1):
//      zc = clamp(depth), disp = RN(k / zc), t = RN(RN(p + 0.5) - disp), target cell
//      floor(t / s) (the division by a power of two is exact), dropped outside [0, ws).
//   2. Alg. 2 over the cells of a row: nearest kept, the lower cell on equal depth: a
//      64-bit atomicMin of (zc bits << 32 | i) into the target cell's key.
//   3. Per full-resolution pixel x in cell j = x / s: a hole if the cell has no key;
//      otherwise its depth is the winner's zc and its color, without interpolation,
//      the pixel at the same place in the winning cell, min(s i + (x - s j), w - 1);
//      with interpolation, the source sampled linearly at texel coordinate u = x + D,
//      D the shift disp interpolated between cell j's and the neighbour's on the side
//      of the pixel centre (weight |x + 0.5 - (s j + s/2)| / s; disp_j alone if that
//      neighbour is a hole or outside the row), clamped to the row's end texels.
//   4. Alg. 3 with Eq. 6 at full resolution over that image: the holes' edges L, R
//      from the mask, the depth gate against zt(L), the weights of Eq. 6 with the
//      exact early exit of FillAcc, the fallback of the base path.
// Every float operation is an explicit round-to-nearest intrinsic, never contracted,
// so the result equals the oracle's byte for byte.
//
// When a band's window and its cells' keys fit shared memory the whole path is one
// band kernel (imb_band in fused.cu: cells, sampling and the fused kernel's band fill
// in shared memory).  Otherwise three launches on the caller's stream after clearing
// the cell keys: cells (one thread per cell), sample (one thread per pixel), and the
// fill: the band fill over the sampled image (fill_only in fused.cu) when a band of
// the window alone fits, else one thread per pixel from global memory.  The cell keys
// and the full-resolution depths of the separate kernels live in handle-owned scratch
// memory.
#include <cuda_runtime.h>

#include <cstdint>

#include "yoro_device.cuh"
#include "yoro_internal.h"

namespace yoro {

namespace {

#ifdef YORO_DEBUG_BOUNDS
__device__ unsigned g_status;  // debug-bounds status word of this file's kernels
__device__ __forceinline__ void yoro_status_record(unsigned code) { atomicOr(&g_status, code); }
#endif

// Steps 1 and 2: one thread per cell.
__global__ void imb_cells_kernel(FrameArgs f, ImbArgs a)
{
    const int w = f.w, ws = a.ws, s = a.div;
    const size_t n = (size_t)ws * (size_t)f.h;
    const uint32_t near_m1 = __float_as_uint(f.near_) - 1u, far_m1 = __float_as_uint(f.far_) - 1u;
    const float inv_s = 1.0f / (float)s;  // a power of two: exact
    for (size_t c = (size_t)blockIdx.x * blockDim.x + threadIdx.x; c < n; c += (size_t)gridDim.x * blockDim.x) {
        const int y = (int)(c / (size_t)ws);
        const int i = (int)(c - (size_t)y * ws);
        const int p = min(s * i + (s >> 1), w - 1);
        const uint32_t zb = clamped_depth_bits(f.depth[(size_t)y * w + p], near_m1, far_m1);
        const float disp = __fdiv_rn(f.k, __uint_as_float(zb));
        const float t = __fsub_rn(__fadd_rn((float)p, 0.5f), disp);
        const float tc = floorf(__fmul_rn(t, inv_s));
        if (tc >= 0.0f && tc < (float)ws && YORO_BOUND(y < f.h, kBadImb))
            atomicMin(&a.cells[(size_t)y * ws + (int)tc], zkey(zb, i));
    }
}

// Step 3: one thread per pixel.  Writes the pixel's color and mask byte, and for a
// reached pixel its depth (the fill's gate); a hole's color is written in step 4.
__global__ void imb_sample_kernel(FrameArgs f, ImbArgs a)
{
    const int w = f.w, ws = a.ws, s = a.div;
    const size_t n = (size_t)w * (size_t)f.h;
    const float inv_s = 1.0f / (float)s;
    for (size_t q = (size_t)blockIdx.x * blockDim.x + threadIdx.x; q < n; q += (size_t)gridDim.x * blockDim.x) {
        const int y = (int)(q / (size_t)w);
        const int x = (int)(q - (size_t)y * w);
        const int j = x / s;
        const unsigned long long* krow = a.cells + (size_t)y * ws;
        const unsigned long long key = krow[j];
        if (key == kEmptyKey) {
            f.mask[q] = 1;
            continue;
        }
        f.mask[q] = 0;
        const uint32_t zb = (uint32_t)(key >> 32);
        a.zt[q] = __uint_as_float(zb);
        const uint32_t* crow = f.color + (size_t)y * w;
        if (!a.interp) {
            const int sx = min(s * (int)(uint32_t)key + (x - s * j), w - 1);
            f.out[q] = YORO_BOUND(sx >= 0, kBadImb) ? crow[sx] : 0u;
            continue;
        }
        const float dj = __fdiv_rn(f.k, __uint_as_float(zb));
        const float off = __fsub_rn(__fadd_rn((float)x, 0.5f), __fadd_rn((float)(s * j), 0.5f * (float)s));
        const int nb = off < 0.0f ? j - 1 : j + 1;
        float d = dj;
        if (off != 0.0f && nb >= 0 && nb < ws && krow[nb] != kEmptyKey) {
            const float dn = __fdiv_rn(f.k, __uint_as_float((uint32_t)(krow[nb] >> 32)));
            d = __fadd_rn(dj, __fmul_rn(__fsub_rn(dn, dj), __fmul_rn(fabsf(off), inv_s)));
        }
        const float u = __fadd_rn((float)x, d);
        uint32_t col;
        if (u <= 0.0f) {
            col = crow[0];
        } else if (u >= (float)(w - 1)) {
            col = crow[w - 1];
        } else {
            const float fl = floorf(u);
            const int i0 = (int)fl;
            const float fr = __fsub_rn(u, fl);
            const uint32_t c0 = crow[i0], c1 = crow[i0 + 1];
            col = 0u;
#pragma unroll
            for (int ch = 0; ch < 4; ++ch) {
                const float v0 = (float)((c0 >> (8 * ch)) & 255u), v1 = (float)((c1 >> (8 * ch)) & 255u);
                const float v = __fadd_rn(v0, __fmul_rn(__fsub_rn(v1, v0), fr));
                col |= (uint32_t)rintf(v) << (8 * ch);
            }
        }
        f.out[q] = col;
    }
}

// Step 4: one thread per pixel; the holes fill from the reached pixels' colors and
// depths (never from another hole), so the writes do not race with the reads.
__global__ void imb_fill_kernel(FrameArgs f, ImbArgs a)
{
    const int w = f.w, h = f.h;
    const size_t n = (size_t)w * (size_t)h;
    for (size_t q = (size_t)blockIdx.x * blockDim.x + threadIdx.x; q < n; q += (size_t)gridDim.x * blockDim.x) {
        if (!f.mask[q]) continue;
        const int v = (int)(q / (size_t)w);
        const int u = (int)(q - (size_t)v * w);
        const uint8_t* mrow = f.mask + (size_t)v * w;
        int L = u - 1;
        while (L >= 0 && mrow[L]) --L;
        int R = u + 1;
        while (R < w && mrow[R]) ++R;
        uint32_t res;
        if (R < w) {
            const int wd = R - L;
            const float d_occ = (L >= 0) ? a.zt[(size_t)v * w + L] : 0.0f;
            FillAcc acc;
            acc.init(__fdiv_rn((float)(R - u), (float)wd));
            const int jhi = min(R + wd, w - 1);
            bool live = true, done = false;
            for (int vv = v - f.halo; vv <= v + f.halo && live; ++vv) {
                if (vv < 0 || vv >= h) continue;
                const size_t ro = (size_t)vv * w;
                for (int st = 0; st <= jhi - R; ++st) {
                    const int j = f.nearest ? R + st : jhi - st;
                    if (f.mask[ro + j]) continue;                // a hole carries no color
                    if (a.zt[ro + j] < d_occ) continue;          // foreground (O2)
                    if (!acc.add(f.out[ro + j])) {               // weight reached exactly 0
                        live = false;
                        break;
                    }
                    if (acc.wrem <= 0.0009765625f && acc.settled(res)) {  // exact early exit
                        live = false;
                        done = true;
                        break;
                    }
                }
            }
            if (!done) res = acc.any() ? acc.result() : f.out[(size_t)v * w + R];
        } else {
            res = (L >= 0) ? f.out[(size_t)v * w + L] : 0u;
        }
        f.out[q] = res;
    }
}

unsigned blocks_for(size_t n, int threads)
{
    size_t b = (n + threads - 1) / threads;
    return (unsigned)(b > 65535u * 8u ? 65535u * 8u : b);
}

}  // namespace

size_t imb_scratch_bytes(int w, int h, int div)
{
    const size_t ws = ((size_t)w + div - 1) / div;
    const size_t keys = ws * (size_t)h * sizeof(unsigned long long);
    return ((keys + 255) & ~(size_t)255) + (size_t)w * h * sizeof(float);
}

ImbArgs imb_args(void* scratch, int w, int h, int div, int interp)
{
    ImbArgs a;
    a.div = div;
    a.interp = interp;
    a.ws = (w + div - 1) / div;
    a.cells = static_cast<unsigned long long*>(scratch);
    const size_t keys = (size_t)a.ws * (size_t)h * sizeof(unsigned long long);
    a.zt = reinterpret_cast<float*>(static_cast<unsigned char*>(scratch) + ((keys + 255) & ~(size_t)255));
    return a;
}

cudaError_t imb_launch(const FrameArgs& f, const ImbArgs& a, const FusedLimits& lim, bool band_fill,
                       cudaStream_t stream)
{
    const size_t nc = (size_t)a.ws * f.h, n = (size_t)f.w * f.h;
    if (n == 0) return cudaSuccess;
    cudaError_t e = cudaMemsetAsync(a.cells, 0xFF, nc * sizeof(unsigned long long), stream);
    if (e != cudaSuccess) return e;
    const int threads = 256;
    imb_cells_kernel<<<blocks_for(nc, threads), threads, 0, stream>>>(f, a);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    imb_sample_kernel<<<blocks_for(n, threads), threads, 0, stream>>>(f, a);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if (band_fill) return fill_only_launch(f, a.zt, lim, stream);
    return fill_pixels_launch(f, a.zt, stream);
}

cudaError_t fill_pixels_launch(const FrameArgs& f, const float* zt, cudaStream_t stream)
{
    const size_t n = (size_t)f.w * f.h;
    if (n == 0) return cudaSuccess;
    ImbArgs a{};
    a.zt = const_cast<float*>(zt);  // the fill reads the depths only
    imb_fill_kernel<<<blocks_for(n, 256), 256, 0, stream>>>(f, a);
    return cudaGetLastError();
}

unsigned imb_status_take()
{
#ifdef YORO_DEBUG_BOUNDS
    unsigned v = 0, z = 0;
    if (cudaMemcpyFromSymbol(&v, g_status, sizeof v) != cudaSuccess ||
        cudaMemcpyToSymbol(g_status, &z, sizeof z) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return v;
#else
    return 0;
#endif
}

}  // namespace yoro
