// yoro_synthesize_noalloc: the global z-buffer path for callers that must not allocate
// device memory.
//
// Some callers cannot call cudaMalloc at the point where they synthesize a frame: a VR
// compositor's per-frame callback cannot afford an allocation that may synchronise the
// device in the middle of a frame, and an engine plugin often runs under a host that
// owns the whole device-memory budget and forbids its plugins from allocating.  This
// entry point serves them with the same kernels as yoro_synthesize_unfused(), but its
// z-buffer is a fixed array in the library's own device memory, created when the module
// is loaded (every GPU that loads the library holds it until the process exits).
#include <cuda_runtime.h>

#include <cmath>
#include <cstddef>
#include <cstdint>
#include <mutex>

#include "yoro.h"
#include "yoro_internal.h"

namespace {

// Largest frame (w * h) this entry point accepts: 2^22 pixels, 32 MiB of keys.
constexpr size_t kNoAllocMaxPixels = (size_t)1 << 22;

// The shared scratch.  In host code this name only stands for the symbol; its device
// address comes from cudaGetSymbolAddress, once per device.
static __device__ __align__(256) unsigned long long g_noalloc_zbuf[kNoAllocMaxPixels];

constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mutex;
unsigned long long* g_noalloc_ptr[kMaxDevices] = {};

// Device address of the scratch on the current device (looked up on first use).
yoro_status noalloc_scratch(unsigned long long** out)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return YORO_ECUDA;
    std::lock_guard<std::mutex> lock(g_noalloc_mutex);
    if (!g_noalloc_ptr[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_zbuf) != cudaSuccess || !p) {
            cudaGetLastError();
            return YORO_ECUDA;
        }
        g_noalloc_ptr[dev] = static_cast<unsigned long long*>(p);
    }
    *out = g_noalloc_ptr[dev];
    return YORO_OK;
}

bool overlaps(const void* a, size_t na, const void* b, size_t nb)
{
    const uintptr_t x = (uintptr_t)a, y = (uintptr_t)b;
    return x < y + nb && y < x + na;
}

}  // namespace

extern "C" {

int yoro_noalloc_max_pixels(void) { return (int)kNoAllocMaxPixels; }

yoro_status yoro_synthesize_noalloc(int w, int h, float fx, float fy, float cx, float cy, float ipd, float near_,
                                    float far_, const void* color, const float* depth, void* out_color,
                                    unsigned char* out_mask, void* stream)
{
    if (w < 0 || h < 0) return YORO_EINVAL;
    for (float v : {fx, fy, cx, cy, ipd, near_, far_})
        if (!std::isfinite(v)) return YORO_EINVAL;
    if (!(fx > 0.0f) || !(ipd >= 0.0f) || !(near_ > 0.0f) || !(far_ > near_)) return YORO_EINVAL;
    const size_t n = (size_t)w * (size_t)h;
    if (n == 0) return YORO_OK;
    if (n > kNoAllocMaxPixels) return YORO_ETOOBIG;
    if (!color || !depth || !out_color || !out_mask) return YORO_EINVAL;
    if (((uintptr_t)color | (uintptr_t)depth | (uintptr_t)out_color) & 3u) return YORO_EALIGN;
    if (overlaps(out_color, 4 * n, color, 4 * n) || overlaps(out_color, 4 * n, depth, 4 * n) ||
        overlaps(out_mask, n, color, 4 * n) || overlaps(out_mask, n, depth, 4 * n) ||
        overlaps(out_mask, n, out_color, 4 * n))
        return YORO_EINVAL;
    unsigned long long* zbuf = nullptr;
    const yoro_status st = noalloc_scratch(&zbuf);
    if (st != YORO_OK) return st;
    yoro::FrameArgs f;
    f.color = (const uint32_t*)color;
    f.depth = depth;
    f.out = (uint32_t*)out_color;
    f.mask = out_mask;
    f.w = w;
    f.h = h;
    f.k = fx * ipd;
    f.near_ = near_;
    f.far_ = far_;
    const double M = ((double)w + 1.5 + (double)f.k / (double)near_) * (1.0 + 1.0 / 1024.0) / 1048576.0;
    f.half_m = M < 0.5 ? (float)(0.5 - M) : 0.0f;
    f.band = 1;
    f.bulk = 0;
    f.halo = 1;     // the paper's kernel: h = 3, farthest column first
    f.nearest = 0;
    // unfused_launch clears the n keys it uses to the empty key before the scatter.
    return yoro::unfused_launch(f, zbuf, (cudaStream_t)stream) == cudaSuccess ? YORO_OK : YORO_ECUDA;
}

}  // extern "C"
