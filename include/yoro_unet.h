/*
 * yoro_unet.h — C ABI of the learned hole inpainter (part of libyoro.so).
 *
 * The paper fills disocclusions with the hand-written Patcher (Sec. Patcher, Alg. 3
 * with Eq. 6); its learned comparison system is a GAN that this library does not
 * reproduce.  The inpainter here is an extension of the method: a 4-level U-Net over
 * 64 x 64 tiles that replaces the Patcher's colors at hole pixels, with the Patcher as
 * its fallback and its yardstick.  Its definition, written out on the CPU, is
 * oracle/unet.py:
 *   input    6 channels per pixel: the plain path's right eye / 255 (the warped colors,
 *            and at holes the Patcher's fill, which the network refines), the hole mask,
 *            near / warped depth (zero at holes), near / source-eye depth;
 *   encoder  levels of 32, 64, 128, 256 channels, two 3x3 convolutions (zero padding)
 *            with ReLU each, 2x2 max pooling between levels;
 *   decoder  nearest 2x upsampling, concatenated after the encoder level's output
 *            (skip channels first), two 3x3 convolutions with ReLU;
 *   output   a 1x1 convolution to 3 channels and a logistic sigmoid.
 * Weights and activations are bfloat16, sums FP32.  The tensor-core kernels sum in
 * another order than the definition, so their results agree with it within the FP32
 * error bound of the sums (then one bfloat16 step where a value sits on a rounding
 * boundary), not bit for bit.
 *
 * Layouts: activations are NHWC bfloat16 (T tiles x H x W x C); weights of a 3x3 layer
 * are K-major bfloat16, Cout rows of 9 * Cin values, k = (3 dy + dx) * Cin + ci.
 * All pointers are device pointers owned by the caller; work is enqueued on the
 * caller's stream (a cudaStream_t as void*).
 */
#ifndef YORO_UNET_H
#define YORO_UNET_H

#include "yoro.h"

#ifdef __cplusplus
extern "C" {
#endif

/*
 * One 3x3 convolution layer on the tensor cores: y = ReLU(conv3x3(x, w) + bias) (relu
 * = 1) or without ReLU (relu = 0), rounded to bfloat16.
 *   x        T x H x W x Cin bfloat16, Cin a multiple of 32 (pad unused channels with 0)
 *   wk       Cout x (9 Cin) bfloat16, K-major as above
 *   bias     Cout floats
 *   y        output NHWC bfloat16 with y_cstride channels per pixel; the layer writes
 *            channels y_coff .. y_coff + Cout - 1 (a decoder's concatenation buffer)
 *   upsample 0: y has T x H x W pixels; 1: y has T x 2H x 2W pixels and every output
 *            pixel is written to its 2 x 2 block (nearest upsampling)
 * Shapes: Cout in {32, 64, 128, 256}; W in {8, 16, 32, 64, 128}; T H W a multiple of
 * 128; when one tile has fewer than 128 pixels, T a multiple of 128 / (H W).  Others:
 * YORO_EINVAL.  y_cstride and y_coff multiples of 8.  YORO_ECUDA if the launch fails.
 * A kernel whose internal wait runs out (it never should) records it for
 * yoro_unet_status().
 */
yoro_status yoro_unet_conv3x3(const void* x, int T, int H, int W, int Cin, const void* wk, const float* bias,
                              void* y, int Cout, int y_cstride, int y_coff, int upsample, int relu,
                              void* cuda_stream);

typedef struct yoro_unet_ctx* yoro_unet;

/* Number of floats in a parameter array: every layer of the definition in order
 * (enc0a, enc0b, enc1a, ..., enc3b, dec2a, dec2b, dec1a, dec1b, dec0a, dec0b, out), each as
 * its weights (Cout x Cin x 3 x 3, or 3 x 32 for the 1x1 output layer, row-major) and
 * then its Cout biases. */
long long yoro_unet_param_count(void);

/*
 * An inpainter on the current device.  params: host floats as above (weights are rounded
 * to bfloat16 here, biases stay FP32); the handle keeps its own copy.  It owns device
 * buffers for max(max_tiles, the tiles of a max_w x max_h frame) 64 x 64 tiles (about
 * 2.9 MB per tile).  NULL if an argument is wrong or an allocation fails.
 */
yoro_unet yoro_unet_create(const float* params, long long n_params, int max_tiles, int max_w, int max_h);
void yoro_unet_destroy(yoro_unet u);

/*
 * The network on T prepared tiles: x is T x 64 x 64 x 32 bfloat16 (the 6 input channels
 * of the definition, channels 6..31 zero, 16-byte aligned); rgb receives T x 64 x 64 x 3
 * floats in [0, 1] (the sigmoid output).  T <= the handle's tile capacity.  Calls on one
 * handle share its buffers: do not overlap them on the GPU.
 */
yoro_status yoro_unet_forward(yoro_unet u, const void* x, int T, float* rgb, void* cuda_stream);

/*
 * Learned inpainting of one synthesized frame, in place.  rgba (w x h RGBA8) holds the
 * right eye from yoro_synthesize_zt(); mask, zt: its hole mask and warped depth;
 * src_depth: the left eye's depth (the source).  The frame is cut into 64 x 64 cells;
 * every cell that holds a hole pixel goes through the network as a 64 x 64 window: the
 * cell itself, or for the last column and row the window shifted inward to end at the
 * frame's edge (so a window never leaves the frame; frames narrower or lower than 64 are
 * padded with zero inputs).  Each hole pixel of the cell takes rint(clamp(c, 0, 1) * 255)
 * per color and alpha 255; reached pixels are not touched.  The tile list is built on the device (nothing
 * is read back).  YORO_ETOOBIG if the frame exceeds the size the handle was created for.
 */
yoro_status yoro_unet_inpaint(yoro_unet u, int w, int h, float near_, void* rgba, const unsigned char* mask,
                              const float* zt, const float* src_depth, void* cuda_stream);

/* One frame of yoro_unet_inpaint_batch(): the arguments of yoro_unet_inpaint(). */
typedef struct {
    int w, h;
    float near_;
    void* rgba;
    const unsigned char* mask;
    const float* zt;
    const float* src_depth;
} yoro_unet_frame;

/*
 * yoro_unet_inpaint() of n frames (each as described there, sizes up to the handle's
 * maximum) in as few passes of the network as its buffers allow: the frames' hole cells
 * form one list, so a pass fills the tensor cores with the cells of several frames.  Each
 * frame's result is the same bytes as yoro_unet_inpaint() of that frame alone (the
 * network treats every cell on its own).  Frames are grouped in order, up to 32 and up to
 * the handle's tile capacity (max(max_tiles, cells of a max_w x max_h frame)) per pass.
 * Every frame is checked before any work is enqueued: the first failing frame's status is
 * returned and nothing runs.  The frames must not overlap one another.
 */
yoro_status yoro_unet_inpaint_batch(yoro_unet u, int n, const yoro_unet_frame* frames, void* cuda_stream);

/*
 * The network inputs of a frame's hole tiles, as yoro_unet_inpaint() builds them (the
 * windows of the hole cells, shifted inward at the last column and row): x_out receives
 * the count tiles (count x 64 x 64 x 32 bfloat16, 16-byte aligned, room for
 * max_out >= the frame's ceil(w/64) * ceil(h/64) tiles), list_host the tiles' indices
 * ty * ceil(w/64) + tx in order and count_host their number.  Synchronises the stream
 * (the host learns the count).  For building training sets.
 */
yoro_status yoro_unet_prepare(yoro_unet u, int w, int h, float near_, const void* rgba, const unsigned char* mask,
                              const float* zt, const float* src_depth, void* x_out, int max_out, int* list_host,
                              int* count_host, void* cuda_stream);

/*
 * Training on the GPU (all in this library's kernels: the forward above, the loss, the
 * backward pass and Adam).  Loss of a batch: the mean over hole pixels and color channels
 * of (s - g)^2, s the network's color and g = ground truth / 255.  The trainer keeps FP32
 * master weights, Adam moments and device buffers for batch_tiles tiles (batch_tiles
 * even).  NULL on a wrong argument or a failed allocation.
 */
typedef struct yoro_unet_trainer_ctx* yoro_unet_trainer;
yoro_unet_trainer yoro_unet_trainer_create(const float* params, long long n_params, int batch_tiles, float lr,
                                           float beta1, float beta2, float eps);
void yoro_unet_trainer_destroy(yoro_unet_trainer t);

/*
 * One step on `tiles` tiles (even, <= batch_tiles): x as for yoro_unet_forward(); gt:
 * tiles x 64 x 64 x 3 bytes (the ground-truth colors); hole: tiles x 64 x 64 bytes (1 =
 * the pixel counts in the loss).  Device pointers.  With lr = 0 the weights do not move
 * and the step's gradients can be read.
 */
yoro_status yoro_unet_train_step(yoro_unet_trainer t, const void* x, const unsigned char* gt,
                                 const unsigned char* hole, int tiles, void* cuda_stream);

/*
 * Copy to host memory, after the work on cuda_stream: what = 0 the master weights, 1 the
 * last step's gradients (yoro_unet_param_count() floats each, the parameter order), 2 the
 * last step's loss (one float).  Synchronises the stream.
 */
yoro_status yoro_unet_trainer_read(yoro_unet_trainer t, int what, float* host_out, void* cuda_stream);

/* The Adam step size of the following steps (>= 0). */
yoro_status yoro_unet_trainer_set_lr(yoro_unet_trainer t, float lr);

/*
 * Synchronise cuda_stream and report the inpainter kernels' status: YORO_ECUDA if CUDA
 * reports an error, YORO_EDEVICE if a kernel gave up an internal wait (the record is
 * read and cleared), else YORO_OK.
 */
yoro_status yoro_unet_status(void* cuda_stream);

#ifdef __cplusplus
}
#endif

#endif /* YORO_UNET_H */
