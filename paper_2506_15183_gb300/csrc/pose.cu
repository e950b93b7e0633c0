// Second-eye synthesis for a general pose of the second eye: Eq. 5 with a general
// M = (VP_left)^-1 VP_right, the eye rotated and offset in any direction, so a pixel
// may leave its row (observation O1 no longer holds).
//
// Reading (the oracle's, step for step): both eyes share the pinhole intrinsics; the
// second eye sits at c (left-eye camera coordinates) with rotation rot, p' = rot (p - c).
//   1. Per source pixel (y, x): zc = clamp(depth) (Alg. 1);
//      p = (((x + 0.5) - cx) zc / fx, ((y + 0.5) - cy) zc / fy, zc); q = p - c;
//      p' = rot q, each component ((r0 q0 + r1 q1) + r2 q2); dropped unless p'.z > 0;
//      target (floor(fx p'.x / p'.z + cx), floor(fy p'.y / p'.z + cy)), dropped outside.
//   2. Alg. 2 over the frame: the nearest p'.z per target, the lower source index
//      y w + x on equal depth: a 64-bit atomicMin of (p'.z bits << 32 | index).
//   3. Gather: the winner's color; p'.z is the target's depth.
//   4. Holes along each row and the Patcher (Alg. 3, Eq. 6) over the gathered image:
//      when a band fits shared memory, the fused kernel's band fill reading the keys
//      itself (fill_keys in fused.cu: steps 3 and 4 in one kernel), else a gather pass
//      and one thread per hole pixel.
// Every float operation is an explicit round-to-nearest intrinsic (IEEE division
// included), never contracted, so the result equals the oracle's byte for byte.
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

__device__ __forceinline__ float dot3(const float* r, float q0, float q1, float q2)
{
    return __fadd_rn(__fadd_rn(__fmul_rn(r[0], q0), __fmul_rn(r[1], q1)), __fmul_rn(r[2], q2));
}

// Steps 1 and 2: one thread per source pixel.
__global__ void pose_scatter_kernel(FrameArgs f, PoseArgs p)
{
    const int w = f.w, h = f.h;
    const size_t n = (size_t)w * (size_t)h;
    const uint32_t near_m1 = __float_as_uint(f.near_) - 1u, far_m1 = __float_as_uint(f.far_) - 1u;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const int y = (int)(i / (size_t)w);
        const int x = (int)(i - (size_t)y * w);
        const float zc = __uint_as_float(clamped_depth_bits(f.depth[i], near_m1, far_m1));
        const float px = __fdiv_rn(__fmul_rn(__fsub_rn(__fadd_rn((float)x, 0.5f), p.cx), zc), p.fx);
        const float py = __fdiv_rn(__fmul_rn(__fsub_rn(__fadd_rn((float)y, 0.5f), p.cy), zc), p.fy);
        const float q0 = __fsub_rn(px, p.c[0]), q1 = __fsub_rn(py, p.c[1]), q2 = __fsub_rn(zc, p.c[2]);
        const float X = dot3(p.rot, q0, q1, q2), Y = dot3(p.rot + 3, q0, q1, q2), Z = dot3(p.rot + 6, q0, q1, q2);
        if (!(Z > 0.0f)) continue;
        const float u = floorf(__fadd_rn(__fdiv_rn(__fmul_rn(p.fx, X), Z), p.cx));
        const float v = floorf(__fadd_rn(__fdiv_rn(__fmul_rn(p.fy, Y), Z), p.cy));
        if (!(u >= 0.0f && u < (float)w && v >= 0.0f && v < (float)h)) continue;
        const size_t o = (size_t)(int)v * w + (int)u;
        if (YORO_BOUND(o < n, kBadPose)) atomicMin(&p.zbuf[o], zkey(__float_as_uint(Z), (int)i));
    }
}

// Step 3: one thread per target pixel.
__global__ void pose_gather_kernel(FrameArgs f, PoseArgs p)
{
    const size_t n = (size_t)f.w * (size_t)f.h;
    for (size_t o = (size_t)blockIdx.x * blockDim.x + threadIdx.x; o < n; o += (size_t)gridDim.x * blockDim.x) {
        const unsigned long long key = p.zbuf[o];
        if (key == kEmptyKey) {
            f.mask[o] = 1;
            continue;
        }
        const uint32_t src = (uint32_t)key;
        f.mask[o] = 0;
        p.zt[o] = __uint_as_float((uint32_t)(key >> 32));
        f.out[o] = YORO_BOUND(src < n, kBadPose) ? f.color[src] : 0u;
    }
}

unsigned blocks_for(size_t n, int threads)
{
    size_t b = (n + threads - 1) / threads;
    return (unsigned)(b > 65535u * 8u ? 65535u * 8u : b);
}

}  // namespace

size_t pose_scratch_bytes(int w, int h)
{
    const size_t n = (size_t)w * (size_t)h;
    return ((n * sizeof(unsigned long long) + 255) & ~(size_t)255) + n * sizeof(float);
}

void pose_bind_scratch(PoseArgs* p, void* scratch, int w, int h)
{
    const size_t n = (size_t)w * (size_t)h;
    p->zbuf = static_cast<unsigned long long*>(scratch);
    p->zt = reinterpret_cast<float*>(static_cast<unsigned char*>(scratch) +
                                     ((n * sizeof(unsigned long long) + 255) & ~(size_t)255));
}

cudaError_t pose_launch(const FrameArgs& f, const PoseArgs& p, const FusedLimits& lim, bool band_fill,
                        cudaStream_t stream)
{
    const size_t n = (size_t)f.w * f.h;
    if (n == 0) return cudaSuccess;
    cudaError_t e = cudaMemsetAsync(p.zbuf, 0xFF, n * sizeof(unsigned long long), stream);
    if (e != cudaSuccess) return e;
    const int threads = 256;
    pose_scatter_kernel<<<blocks_for(n, threads), threads, 0, stream>>>(f, p);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    // a band fits shared memory: the band fill reads the keys itself (gather included)
    if (band_fill) return fill_keys_launch(f, p.zbuf, lim, stream);
    pose_gather_kernel<<<blocks_for(n, threads), threads, 0, stream>>>(f, p);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    return fill_pixels_launch(f, p.zt, stream);
}

unsigned pose_status_take()
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
