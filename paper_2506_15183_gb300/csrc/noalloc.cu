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

#include <cstddef>
#include <cstdint>

#include "yoro.h"
#include "yoro_internal.h"

namespace {

// Largest frame (w * h) this entry point accepts: 2^22 pixels, 32 MiB of keys.
constexpr size_t kNoAllocMaxPixels = (size_t)1 << 22;

// The shared scratch.  In host code this name only stands for the symbol; its device
// address comes from cudaGetSymbolAddress.
static __device__ __align__(256) unsigned long long g_noalloc_zbuf[kNoAllocMaxPixels];

// Device address of the scratch on the current device.  Looked up on every call: the
// lookup allocates nothing, and an address kept from an earlier call could be stale
// after cudaDeviceReset() (the module, and with it the array, is loaded again).  The
// first lookup on a device loads the library's module there.
yoro_status noalloc_scratch(unsigned long long** out)
{
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_zbuf) != cudaSuccess || !p) {
        cudaGetLastError();
        return YORO_ECUDA;
    }
    *out = static_cast<unsigned long long*>(p);
    return YORO_OK;
}

}  // namespace

extern "C" {

int yoro_noalloc_max_pixels(void) { return (int)kNoAllocMaxPixels; }

yoro_status yoro_synthesize_noalloc(int w, int h, float fx, float fy, float cx, float cy, float ipd, float near_,
                                    float far_, const void* color, const float* depth, void* out_color,
                                    unsigned char* out_mask, void* stream)
{
    // the camera checks of yoro_create and the pointer checks of yoro_synthesize
    if (!yoro::camera_valid(w, h, fx, fy, cx, cy, ipd, near_, far_)) return YORO_EINVAL;
    const size_t n = (size_t)w * (size_t)h;
    if (n == 0) return YORO_OK;
    if (n > kNoAllocMaxPixels) return YORO_ETOOBIG;
    yoro::FrameArgs f;
    const int chk = yoro::checked_frame(w, h, fx * ipd, near_, far_, color, depth, out_color, out_mask, &f);
    if (chk != YORO_OK) return (yoro_status)chk;
    unsigned long long* zbuf = nullptr;
    const yoro_status st = noalloc_scratch(&zbuf);
    if (st != YORO_OK) return st;
    // unfused_launch clears the n keys it uses to the empty key before the scatter.
    return yoro::unfused_launch(f, zbuf, (cudaStream_t)stream) == cudaSuccess ? YORO_OK : YORO_ECUDA;
}

}  // extern "C"
