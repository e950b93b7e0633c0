// Host/device interface between the C ABI (api.cu) and the kernel launchers.
#pragma once

#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>

namespace yoro {

// Debug-bounds build (-DYORO_DEBUG_BOUNDS): YORO_BOUND(cond, code) is true when cond
// holds; otherwise it ORs `code` into the translation unit's device status word and is
// false, and the caller skips the access it guards.  Nothing traps.  In release builds
// it is the constant true and costs nothing.
#ifdef YORO_DEBUG_BOUNDS
#define YORO_BOUND(cond, code) ((cond) ? true : (yoro_status_record(code), false))
#else
#define YORO_BOUND(cond, code) true
#endif

// Codes of the status word (bits).
constexpr unsigned kBadScatter = 1u;   // P1: depth load or target word outside the window
constexpr unsigned kBadResolve = 2u;   // P2: window word, gather or output pixel out of range
constexpr unsigned kBadHoles = 4u;     // P3a/P3b: hole bookkeeping or fill index out of range
constexpr unsigned kBadUnfused = 8u;   // the z-buffer kernels
constexpr unsigned kSelfTest = 16u;    // yoro_debug_selftest
constexpr unsigned kBadImb = 32u;      // row-downsampled intermediate buffer kernels
constexpr unsigned kBadPose = 64u;     // general-pose reprojection kernels

// One frame as the kernels see it.  color/out are RGBA8 pixels read as uint32.
struct FrameArgs {
    const uint32_t* color;
    const float* depth;
    uint32_t* out;
    uint8_t* mask;
    int w, h;
    float k;      // fx * ipd, rounded once to binary32 on the host
    float near_, far_;
    float half_m; // 0.5 - M: decision margin of the approximate disparity (host bound)
    int band;     // rows per CTA work item
    int bulk;     // 1: rows are 16-byte aligned (w % 4 == 0), bulk copies + vector stores
    int halo;     // Patcher kernel rows on each side of v: kernel height 2 halo + 1 (default 1)
    int nearest;  // 1: kernel columns nearest first (R up); 0: farthest first (default)
    float* zt_out;  // optional (fused default kernel only): warped depth per pixel, 0 at holes
};

// Up to kMaxBatch frames travel in the kernel's parameter space (< 32 KB).
constexpr int kMaxBatch = 256;

struct BatchArgs {
    int n;
    int total_items;
    int max_band;                   // tallest band of the launch (sizes shared memory)
    int item_start[kMaxBatch + 1];  // prefix sum of bands per frame
    FrameArgs f[kMaxBatch];
};

struct FusedLimits {
    int sms;
    int smem_per_block;
    int smem_per_sm;
    int max_width;  // widest frame whose rows fit the fused kernel's shared memory
};

// Launch shape of one frame: rows per CTA, and whether two CTAs share an SM.
struct FusedShape {
    int band;
    int two_per_sm;
};

// fused.cu
int fused_wpad(int w);
size_t fused_smem_bytes(int wpad, int band, int halo = 1);
cudaError_t fused_configure(int device, FusedLimits* lim);
FusedShape fused_shape(const FusedLimits& lim, int w, int h, int halo = 1);
int fused_max_band(const FusedLimits& lim, int w, int halo = 1);
cudaError_t fused_launch(const FrameArgs& f, const FusedLimits& lim, int two_per_sm, cudaStream_t stream);
// zt: the instantiation that writes each frame's warped depth where its zt_out is set.
cudaError_t fused_launch_batch(const BatchArgs& a, int wmax, const FusedLimits& lim, cudaStream_t stream,
                               bool zt = false);

// api.cu: the camera checks of yoro_create, and the status yoro_last_create_error reports.
bool camera_valid(int w, int h, float fx, float fy, float cx, float cy, float ipd, float near_, float far_);
void set_last_create_error(int status);
// The pointer checks of every device-pointer entry point (null, 4-byte alignment,
// overlap of outputs with inputs) and the frame description with its disparity
// decision margin, for the paper's default kernel; returns a yoro_status.
int checked_frame(int w, int h, float k, float near_, float far_, const void* color, const float* depth, void* out,
                  unsigned char* mask, FrameArgs* f);

// Status words of the debug-bounds build (0 in release builds): read and cleared,
// after the caller synchronised.  fused.cu also launches the self-test kernel.
unsigned fused_status_take();
unsigned unfused_status_take();
cudaError_t debug_selftest_launch(cudaStream_t stream);
bool debug_bounds_built();

// unfused.cu: separate kernels around a global z-buffer of h*w keys.
cudaError_t unfused_launch(const FrameArgs& f, unsigned long long* zbuf, cudaStream_t stream);

// The row-downsampled intermediate buffer (imbuffer.cu): div source pixels per cell
// (1, 2, 4, 8 or 16), linear interpolation of the shift and the color when interp.
struct ImbArgs {
    unsigned long long* cells;  // h * ws keys (clamped depth bits << 32 | source cell)
    float* zt;                  // h * w depths of the reached pixels
    int div, interp, ws;
};
size_t imb_scratch_bytes(int w, int h, int div);
ImbArgs imb_args(void* scratch, int w, int h, int div, int interp);
// band_fill: the frame's band window fits shared memory (fused_ok), so the holes are
// filled by fill_only_launch; otherwise by one thread per pixel from global memory.
cudaError_t imb_launch(const FrameArgs& f, const ImbArgs& a, const FusedLimits& lim, bool band_fill,
                       cudaStream_t stream);
// The fused kernel's hole fill (P3) over a frame resolved in global memory: reached
// colors in f.out, their depths in zt, the hole mask in f.mask.
cudaError_t fill_only_launch(FrameArgs f, const float* zt, const FusedLimits& lim, cudaStream_t stream);
// The same fill read straight from a frame-wide z-buffer of 64-bit keys (depth bits above
// the source index, ~0 at holes): also writes the reached pixels' colors (gathered from
// f.color) and the hole mask.
cudaError_t fill_keys_launch(FrameArgs f, const unsigned long long* keys, const FusedLimits& lim, cudaStream_t stream);
// The holes of a frame resolved in global memory (colors in f.out, depths in zt, mask
// in f.mask), one thread per pixel: for frames too wide for a band window.
cudaError_t fill_pixels_launch(const FrameArgs& f, const float* zt, cudaStream_t stream);

// General second-eye pose (pose.cu): p' = rot (p - c) with the shared intrinsics.
struct PoseArgs {
    float fx, fy, cx, cy;
    float rot[9];               // row-major
    float c[3];                 // second eye position in left-eye camera coordinates
    unsigned long long* zbuf;   // h * w keys (p'.z bits << 32 | source index)
    float* zt;                  // h * w depths of the reached targets
};
size_t pose_scratch_bytes(int w, int h);
void pose_bind_scratch(PoseArgs* p, void* scratch, int w, int h);
cudaError_t pose_launch(const FrameArgs& f, const PoseArgs& p, const FusedLimits& lim, bool band_fill,
                        cudaStream_t stream);
unsigned pose_status_take();

// The intermediate buffer in one band kernel (cell keys, sampling and fill in shared
// memory): the tallest band whose window and cell keys fit (0 if none), and the launch.
size_t imb_band_smem_bytes(int w, int band, int halo, int div);
int imb_band_max(const FusedLimits& lim, int w, int halo, int div);
cudaError_t imb_band_launch(FrameArgs f, int div, int interp, const FusedLimits& lim, cudaStream_t stream);
unsigned imb_status_take();

}  // namespace yoro
