/*
 * yoro.h — C ABI of the GB300 second-eye synthesis library (libyoro.so).
 *
 * Given the rendered LEFT eye of a stereo pair (RGBA8 color and FP32 linear
 * view-space depth), the library produces the RIGHT eye (RGBA8) and a hole mask,
 * following "You Only Render Once" (YORO):
 *   1. disparity per source pixel (Sec. Reprojector, Alg. 1 with Eq. 5 in closed
 *      form for a parallel-axis pinhole pair): zc = clamp(z, near, far),
 *      disp = (fx * ipd) / zc, target column xt = floor(x + 0.5 - disp);
 *   2. forward warp with the nearest source kept per target (Alg. 2; on equal
 *      depth the lowest source column wins);
 *   3. gather: a reached target takes its source's four bytes (Alg. 3, non-hole
 *      branch);
 *   4. disocclusion tracking (Sec. Reprojector, strategy (b)): nearest reached
 *      column on each side of a hole;
 *   5. hole fill (Sec. Patcher, Alg. 3 with the weight of Eq. 6) over rows
 *      v-1..v+1 on the background side, foreground candidates skipped (O2).
 * Every step runs in the library's CUDA kernels (sm_103a); all arithmetic is
 * IEEE binary32 with no fused multiply-add, so the output is a deterministic
 * function of the inputs.
 *
 * Conventions shared by every entry point:
 *   - Images are tightly packed, row-major, row 0 at the top. color / out_color
 *     hold h*w*4 bytes (R, G, B, A per pixel), depth holds h*w floats,
 *     out_hole_mask holds h*w bytes (1 = the pixel was a hole before the fill,
 *     0 = reached by a source pixel).
 *   - Pointers named device pointers must point to memory of the device that was
 *     current when the handle was created; color/out_color/depth need 4-byte
 *     alignment.  16-byte aligned pointers with w % 4 == 0 take the bulk-copy fast
 *     path; other layouts are accepted and take a slower element-wise path.
 *   - The caller owns every image buffer.  Outputs must not overlap inputs.
 *   - Work is enqueued on the caller's CUDA stream (a cudaStream_t passed as
 *     void*, NULL = the legacy default stream) and returns before it finishes.
 *     Argument errors are reported synchronously; errors raised while the kernels
 *     run surface from yoro_stream_status() or from the caller's own stream
 *     synchronisation.
 *   - A handle may be used from one host thread at a time.  Calls on different
 *     streams may overlap on the GPU except where an entry point says it uses
 *     handle-owned scratch memory.
 */
#ifndef YORO_H
#define YORO_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct yoro_ctx* yoro_handle;

typedef enum {
    YORO_OK = 0,
    YORO_EINVAL = 1,   /* bad argument: null pointer, size, camera parameter, wrong device */
    YORO_EALIGN = 2,   /* a pointer is not 4-byte aligned                                 */
    YORO_ENOMEM = 3,   /* a device or pinned-host allocation failed                       */
    YORO_ECUDA = 4,    /* a CUDA runtime call or kernel launch failed                     */
    YORO_EDEVICE = 5,  /* a kernel of the debug-bounds build skipped an out-of-range access */
    YORO_ETOOBIG = 6,  /* the frame exceeds a limit of the requested entry point          */
    YORO_ETIMEOUT = 7, /* a wait with a time limit ran out (yoro_server_drain)           */
    YORO_ECANCELED = 8 /* the request was cancelled before it ran (yoro_server_cancel)   */
} yoro_status;

/* One frame of a batch (yoro_synthesize_batch).  All pointers are device pointers. */
typedef struct {
    int w, h;
    float fx, fy, cx, cy, ipd, near_, far_;
    const void* color;           /* h*w*4 bytes RGBA8, left eye          */
    const float* depth;          /* h*w floats, linear view-space depth  */
    void* out_color;             /* h*w*4 bytes RGBA8, right eye         */
    unsigned char* out_hole_mask;/* h*w bytes                            */
} yoro_frame;

/* Variants of the Patcher's kernel (Sec. Patcher).  yoro_create() takes the paper's
 * kernel: height 3, columns visited farthest first. */
typedef struct {
    int kernel_rows;   /* kernel height h: odd, 1..15; rows v-(h-1)/2 .. v+(h-1)/2 (paper: 3) */
    int nearest_first; /* 0: each row's columns from min(R + w, W - 1) down to R, the farthest
                          first (the paper's order, mirrored to a left-eye source);
                          1: from R up, the nearest first */
} yoro_options;

/*
 * Create a synthesis context for w x h frames of a stereo camera.
 *   fx, fy, cx, cy: pinhole intrinsics in pixels (shared by both eyes).  Only fx
 *     enters the result: with parallel axes and a horizontal baseline the row is
 *     unchanged and cx cancels (Eq. 5 in closed form).
 *   ipd: eye separation in scene units (>= 0); the right eye sits at +ipd along x.
 *   near_, far_: depth clamp, 0 < near_ < far_ (the camera planes of Eq. 3).  A
 *     depth that is not a positive finite number is treated as far_.
 * Requires w >= 0, h >= 0, w * h < 2^31, fx > 0, all parameters finite.
 * Records the current device; allocates no device memory.
 * Returns NULL on error; yoro_last_create_error() then tells why.
 */
yoro_handle yoro_create(int w, int h, float fx, float fy, float cx, float cy, float ipd,
                        float near_, float far_);

/* yoro_create() with a Patcher kernel variant (opt may be NULL: the paper's kernel).  The
 * handle's synthesize calls (fused, unfused and host) use it; a frame whose band of one
 * row with its kernel rows does not fit shared memory takes the global z-buffer path.
 * Batch and no-alloc calls always use the paper's kernel.  Returns NULL with
 * YORO_EINVAL for an even or out-of-range kernel_rows or a nearest_first other than
 * 0 or 1. */
yoro_handle yoro_create_ex(int w, int h, float fx, float fy, float cx, float cy, float ipd, float near_,
                           float far_, const yoro_options* opt);

/*
 * yoro_create_ex() with the Reprojector's row-downsampled intermediate buffer
 * (strategies (c) and (d) of the paper: an ImBuffer at 1/2 .. 1/16 of the per-eye
 * resolution, "sampled based on linear interpolation of the distance shifted").  The
 * paper gives their intent only; the reading implemented:
 *   imbuffer_div s in {1, 2, 4, 8, 16}: each row is reprojected in cells of s source
 *     pixels (ceil(w / s) per row): a cell's depth is that of its pixel
 *     min(s i + s/2, w - 1), its target cell floor(((p + 0.5) - k / zc) / s), the
 *     nearest source cell kept per target cell, which records its shift k / zc;
 *   interpolate 0: a right-eye pixel copies the pixel at the same place in its cell's
 *     winning cell; 1: the source is sampled linearly (per channel, rounded half to
 *     even) at x + D, D the shift interpolated between the pixel's cell and the
 *     neighbouring cell on the side of the pixel centre, clamped to the row's ends;
 *   a pixel whose cell no source cell reaches is a hole, filled by the Patcher at full
 *   resolution (the handle's kernel variant) from the reached pixels, whose depth is
 *   their winning cell's.
 * s = 1 without interpolation is the base path.  Every synthesize call of the handle
 * (fused, unfused, host, mapped) takes this path when s > 1 or interpolate = 1: one
 * band kernel when a band of rows with its cells fits shared memory, else (and for
 * yoro_synthesize_unfused) three launches around handle-owned scratch memory
 * (8 ceil(w/s) h + 4 w h bytes, allocated on the first such call); same result.
 * Returns NULL with YORO_EINVAL for another s or interpolate, and as yoro_create_ex()
 * otherwise.
 */
yoro_handle yoro_create_imb(int w, int h, float fx, float fy, float cx, float cy, float ipd, float near_,
                            float far_, const yoro_options* opt, int imbuffer_div, int interpolate);

/*
 * A context for a general pose of the second eye (Eq. 5 with a general
 * M = (VP_left)^-1 VP_right): rotated and offset in any direction, so that pixels may
 * leave their row.  Both eyes share the pinhole intrinsics fx, fy, cx, cy (all used).
 * rotation: 9 floats, row-major, and position: 3 floats, the second eye's rotation R and
 * centre c in left-eye camera coordinates: a point p seen by the left eye is at
 * R (p - c) for the second eye (R = I, c = (ipd, 0, 0) is yoro_create's stereo pair).
 * Per source pixel: the clamped depth zc (as yoro_create), p = (((x + 0.5) - cx) zc / fx,
 * ((y + 0.5) - cy) zc / fy, zc), p' = R (p - c) with each component ((r0 q0 + r1 q1) + r2 q2),
 * dropped unless p'.z > 0, target (floor(fx p'.x / p'.z + cx), floor(fy p'.y / p'.z + cy));
 * per target the nearest p'.z is kept, the lower source index y w + x on equal depth;
 * holes are found along the rows and filled by the Patcher (opt: its kernel variant),
 * with p'.z as the depths.  Every synthesize call of the handle takes this path: three
 * launches around handle-owned scratch memory (12 w h bytes, allocated on the first
 * call).  Returns NULL with YORO_EINVAL for NULL or non-finite rotation / position, a
 * non-positive fy, and as yoro_create_ex() otherwise.
 */
yoro_handle yoro_create_pose(int w, int h, float fx, float fy, float cx, float cy, const float* rotation,
                             const float* position, float near_, float far_, const yoro_options* opt);

/* Status of the last yoro_create*() call on the calling thread (YORO_OK after a
 * success). */
yoro_status yoro_last_create_error(void);

/* Release the handle and the device memory it owns.  NULL is accepted.  Pending work
 * that uses handle-owned scratch must have finished (synchronise first). */
void yoro_destroy(yoro_handle h);

/*
 * Synthesize the right eye of one frame (all five steps, one fused kernel that
 * keeps each band of rows in shared memory).
 *   color_rgba8, depth_f32: device inputs (left eye).
 *   out_color_rgba8, out_hole_mask: device outputs (right eye).
 *   cuda_stream: cudaStream_t or NULL.
 * Uses no scratch memory for widths up to yoro_max_fused_width(); wider frames
 * run the global z-buffer path of yoro_synthesize_unfused() (see there).
 * An empty frame (w * h == 0) returns YORO_OK without launching anything.
 */
yoro_status yoro_synthesize(yoro_handle h, const void* color_rgba8, const float* depth_f32,
                            void* out_color_rgba8, unsigned char* out_hole_mask, void* cuda_stream);

/*
 * yoro_synthesize() that also writes the warped depth: out_zt (h*w floats, device,
 * 4-byte aligned, not overlapping any other buffer) receives, at every reached pixel,
 * the clamped depth of the source that won it (Alg. 2's stored depth), and 0 at holes.
 * The learned inpainter (yoro_unet.h) takes it as an input channel.  Only for handles
 * of yoro_create() (the paper's Patcher, no variant) whose frames take the fused
 * kernel (w <= yoro_max_fused_width()); YORO_EINVAL otherwise.
 */
yoro_status yoro_synthesize_zt(yoro_handle h, const void* color_rgba8, const float* depth_f32,
                               void* out_color_rgba8, unsigned char* out_hole_mask, float* out_zt,
                               void* cuda_stream);

/*
 * Same result as yoro_synthesize(), computed by separate kernels around a global
 * z-buffer of h*w 64-bit keys (depth bits << 32 | source column) that the handle
 * allocates on first use and keeps.  Works for any width.  Calls that share a
 * handle must not overlap on the GPU (they share the z-buffer).
 */
yoro_status yoro_synthesize_unfused(yoro_handle h, const void* color_rgba8, const float* depth_f32,
                                    void* out_color_rgba8, unsigned char* out_hole_mask,
                                    void* cuda_stream);

/*
 * yoro_synthesize() for HOST buffers: copies color and depth to device staging
 * owned by the handle (allocated on first use), runs the fused kernel, and copies
 * the right eye and mask back, all on cuda_stream.  Page-locked (pinned) host
 * buffers give asynchronous copies; the call returns before the copies finish,
 * so the caller synchronises the stream before reading the outputs.  Calls that
 * share a handle must not overlap on the GPU (they share the staging).
 */
yoro_status yoro_synthesize_host(yoro_handle h, const void* host_color_rgba8, const float* host_depth_f32,
                                 void* host_out_color_rgba8, unsigned char* host_out_hole_mask,
                                 void* cuda_stream);

/*
 * yoro_synthesize() on HOST buffers without staging copies (zero copy): the kernels load
 * the left eye from and store the right eye and mask to page-locked host memory that is
 * mapped into the device address space (cudaHostAlloc / cudaHostRegister with mapping;
 * on systems with unified addressing every page-locked allocation is), over the
 * host-device link (NVLink-C2C on Grace systems).  Each pointer is checked with
 * cudaPointerGetAttributes: anything else returns YORO_EINVAL before any launch.  Same
 * layout, alignment and result as yoro_synthesize; the L2 bulk prefetch of the inputs is
 * not used.  Returns before the kernel finishes; synchronise the stream before reading.
 */
yoro_status yoro_synthesize_mapped(yoro_handle h, const void* host_color_rgba8, const float* host_depth_f32,
                                   void* host_out_color_rgba8, unsigned char* host_out_hole_mask,
                                   void* cuda_stream);

/*
 * Synthesize n independent frames of possibly different sizes and cameras in one
 * persistent kernel launch (the same five steps per frame; results equal n calls of
 * yoro_synthesize).  frames: host array of n descriptors with device pointers; up to
 * 256 frames share one launch (larger n takes several).  Needs no handle and allocates
 * no device memory.  Returns YORO_ETOOBIG if a frame is wider than
 * yoro_max_fused_width() or if n exceeds 4096.
 */
yoro_status yoro_synthesize_batch(int n, const yoro_frame* frames, void* cuda_stream);

/*
 * Autotuner of yoro_synthesize_batch (a library service; the paper has no counterpart).
 * Runs the batch `frames` (same arguments and contract as yoro_synthesize_batch) at a few
 * band heights (rows per work item: the tallest that fits shared memory for the widest
 * frame, a few just below it, and about 3/4, 1/2, 1/3 and 1/4 of it; the shorter ones
 * run two CTAs of 512 threads per SM), `reps` timed launches each after one untimed one
 * (CUDA events on cuda_stream), and keeps the fastest for this device and this widest
 * width: later yoro_synthesize_batch launches on the device whose widest frame has that
 * width use it.  Writes the chosen band to *out_band (if not NULL).  Every candidate
 * computes the same outputs, so the frames' outputs hold the result when it returns.
 * Synchronises cuda_stream.  1 <= reps <= 1000, n >= 1 with at least one non-empty frame.
 * Returns the errors of yoro_synthesize_batch; the tuned table is left unchanged on error.
 */
yoro_status yoro_tune_batch(int n, const yoro_frame* frames, int reps, void* cuda_stream, int* out_band);

/* Rows per work item that yoro_synthesize_batch uses on the current device for the
 * widest frame of a launch, w pixels: the tuned height, else the tallest that fits
 * shared memory.  Narrower frames of the launch take as many rows as fit the same shared
 * memory with their own row length.  0 if w < 1, w > yoro_max_fused_width() or the
 * device cannot be queried. */
int yoro_batch_band(int w);

/* Forget every tuned band height (all devices). */
void yoro_reset_tuning(void);

/*
 * Synchronise cuda_stream and report whether work on it failed: YORO_ECUDA if the
 * stream or the runtime reports a CUDA error; in the debug-bounds build YORO_EDEVICE if
 * a kernel of this library recorded a skipped access since the last call (the record
 * is cleared by reading it; it is device-wide, not per stream); else YORO_OK.  h may be
 * NULL (batch launches have no handle).
 */
yoro_status yoro_stream_status(yoro_handle h, void* cuda_stream);

/*
 * 1 if this library is the debug-bounds build, else 0.  That build compiles the same
 * kernels with a range check in front of every shared- and global-memory access whose
 * index is computed (source and target columns, window rows, hole positions, z-buffer
 * keys); an access that fails its check is skipped, never made, and a code is OR-ed into
 * a device status word that yoro_stream_status() reports.  No kernel traps.  The release
 * build compiles the checks away.
 */
int yoro_debug_bounds_enabled(void);

/*
 * Launch, on cuda_stream, a one-warp kernel that records a code in the debug-bounds
 * status word and touches no memory, so that a caller can see the reporting path work:
 * yoro_stream_status() then returns YORO_EDEVICE once.  In the release build the kernel
 * records nothing.  YORO_ECUDA if the launch fails.
 */
yoro_status yoro_debug_selftest(void* cuda_stream);

/*
 * yoro_synthesize_unfused() without a handle and without allocating device memory, for
 * callers that must not call cudaMalloc where they synthesize: a compositor's per-frame
 * callback (an allocation may synchronise the device mid-frame) or a plugin whose host
 * owns the device-memory budget.  The paper has no counterpart; this is a library
 * service.  Same camera parameters as yoro_create() and the same device pointers and
 * layout as yoro_synthesize(); same result.
 * The z-buffer is one array in the library's device memory, 2^22 keys (32 MiB), held by
 * every GPU that loads the library until the process exits: frames with w * h greater
 * than yoro_noalloc_max_pixels() are rejected with YORO_ETOOBIG.  Every call looks up
 * that array's device address (cudaGetSymbolAddress, no allocation), so the address
 * stays right after a cudaDeviceReset(); the first call on a device also loads the
 * library's module there.  Every call clears the part of the array it uses on
 * cuda_stream, and every call on every stream shares the array, so calls that could
 * overlap on the GPU race: serialise them (one stream, or events).
 */
yoro_status yoro_synthesize_noalloc(int w, int h, float fx, float fy, float cx, float cy, float ipd,
                                    float near_, float far_, const void* color_rgba8, const float* depth_f32,
                                    void* out_color_rgba8, unsigned char* out_hole_mask, void* cuda_stream);

/* Largest w * h that yoro_synthesize_noalloc() accepts (4,194,304). */
int yoro_noalloc_max_pixels(void);

/* Widest frame the fused single-kernel path handles on the current device. */
int yoro_max_fused_width(void);

/* Static English description of a status code. */
const char* yoro_status_string(yoro_status s);

#ifdef __cplusplus
}
#endif

#endif /* YORO_H */
