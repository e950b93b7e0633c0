// Unfused second-eye synthesis: separate kernels around a global z-buffer.
//
// Works for any frame width (the fused kernel keeps four rows of keys in shared
// memory, which bounds its width).  Three launches on the caller's stream:
//   1. clear the z-buffer to the empty key (cudaMemsetAsync);
//   2. scatter: per source pixel, disparity (Alg. 1 closed form) and a 64-bit
//      atomicMin of (depth bits << 32 | source column) into zbuf[y][xt] (Alg. 2,
//      nearest kept; ties to the lowest source column);
//   3. resolve + fill: per target pixel, the gather of a reached pixel, or for a
//      hole the edges L/R, the occluder depth and the depth-gated weighted fill of
//      Alg. 3 / Eq. 6 over rows v-1..v+1, reading keys and source colors from
//      global memory.
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

__global__ void scatter_kernel(FrameArgs f, unsigned long long* __restrict__ zbuf)
{
    const size_t n = (size_t)f.w * (size_t)f.h;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const int y = (int)(i / (size_t)f.w);
        const int x = (int)(i - (size_t)y * f.w);
        uint32_t zb;
        const int xt = disparity_target(f.depth[i], __fadd_rn((float)x, 0.5f), f.k, __float_as_uint(f.near_) - 1u,
                                        __float_as_uint(f.far_) - 1u, f.half_m, zb);
        if (xt >= 0 && xt < f.w && YORO_BOUND(y < f.h, kBadUnfused))
            atomicMin(&zbuf[(size_t)y * f.w + xt], zkey(zb, x));
    }
}

__device__ __forceinline__ uint32_t key_color(const FrameArgs& f, int row, unsigned long long key)
{
    // the key's low word is a source column of the row (checked in the debug-bounds build)
    const uint32_t c = (uint32_t)key;
    return YORO_BOUND(c < (uint32_t)f.w && row >= 0 && row < f.h, kBadUnfused) ? f.color[(size_t)row * f.w + c] : 0u;
}

__global__ void resolve_fill_kernel(FrameArgs f, const unsigned long long* __restrict__ zbuf)
{
    const size_t n = (size_t)f.w * (size_t)f.h;
    const int w = f.w;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const int v = (int)(i / (size_t)w);
        const int u = (int)(i - (size_t)v * w);
        const unsigned long long* zr = zbuf + (size_t)v * w;
        const unsigned long long key = zr[u];
        if (key != kEmptyKey) {
            f.out[i] = key_color(f, v, key);
            f.mask[i] = 0;
            continue;
        }
        f.mask[i] = 1;
        int L = u - 1;
        while (L >= 0 && zr[L] == kEmptyKey) --L;
        int R = u + 1;
        while (R < w && zr[R] == kEmptyKey) ++R;
        uint32_t res;
        if (R < w) {
            const int wd = R - L;
            const float d_occ = (L >= 0) ? __uint_as_float((uint32_t)(zr[L] >> 32)) : 0.0f;
            FillAcc acc;
            acc.init(__fdiv_rn((float)(R - u), (float)wd));
            const int jhi = min(R + wd, w - 1);
            bool live = true, done = false;
            for (int vv = v - f.halo; vv <= v + f.halo && live; ++vv) {
                if (vv < 0 || vv >= f.h) continue;
                const unsigned long long* zq = zbuf + (size_t)vv * w;
                for (int s = 0; s <= jhi - R; ++s) {
                    const int j = f.nearest ? R + s : jhi - s;
                    const unsigned long long kq = zq[j];
                    if (kq == kEmptyKey) continue;
                    if (__uint_as_float((uint32_t)(kq >> 32)) < d_occ) continue;
                    if (!acc.add(key_color(f, vv, kq))) {  // weight reached exactly 0
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
            if (!done) res = acc.any() ? acc.result() : key_color(f, v, zr[R]);
        } else {
            res = (L >= 0) ? key_color(f, v, zr[L]) : 0u;
        }
        f.out[i] = res;
    }
}

}  // namespace

cudaError_t unfused_launch(const FrameArgs& f, unsigned long long* zbuf, cudaStream_t stream)
{
    const size_t n = (size_t)f.w * (size_t)f.h;
    cudaError_t e = cudaMemsetAsync(zbuf, 0xFF, n * sizeof(unsigned long long), stream);
    if (e != cudaSuccess) return e;
    const int threads = 256;
    size_t blocks = (n + threads - 1) / threads;
    if (blocks > 65535u * 8u) blocks = 65535u * 8u;
    scatter_kernel<<<(unsigned)blocks, threads, 0, stream>>>(f, zbuf);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    resolve_fill_kernel<<<(unsigned)blocks, threads, 0, stream>>>(f, zbuf);
    return cudaGetLastError();
}

unsigned unfused_status_take()
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
