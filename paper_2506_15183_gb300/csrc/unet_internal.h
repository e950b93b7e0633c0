// Internal interface of the learned inpainter (unet.cu, unet_train.cu).
#pragma once

#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>

namespace yoro {

// Parameters of the network: 14 3x3 layers (enc0a, enc0b, ..., enc3b, dec2a, dec2b, dec1a,
// dec1b, dec0a, dec0b) and the 1x1 output layer, in the order of the definition.
struct UnetLayer {
    int cin, cout, cin_pad;
    uint16_t* wk;  // device, K-major bfloat16
    float* bias;   // device
};

struct UnetNet {
    UnetLayer conv[14];
    float* wout;  // device: 3 x 32 (bfloat16 values as floats), then 3 biases
    int max_tiles;
    // activations, NHWC bfloat16, for max_tiles tiles
    uint16_t *in0, *e0a, *cat0, *p0, *e1a, *cat1, *p1, *e2a, *cat2, *p2, *e3a, *d2a, *d1a, *d0a, *d0b;
    int *flags, *list, *count;
    int max_grid_tiles;  // capacity of flags / list
};

size_t unet_param_count();
void unet_layer_dims(int i, int* cin, int* cout);
UnetNet* unet_create(const float* params, size_t n_params, int max_tiles, int max_grid_tiles);
void unet_free(UnetNet* n);
cudaError_t unet_run(UnetNet* n, int T, const int* count, cudaStream_t s);
cudaError_t unet_conv3x3(const void* x, int T, int H, int W, int Cin, const void* wk, const float* bias, void* y,
                         int Cout, int y_cstride, int y_coff, int upsample, int relu, cudaStream_t stream,
                         const int* count = nullptr);
// The output layer (1x1 convolution, sigmoid) of T tiles' d0b activations into rgb (T x 64 x 64 x 3).
cudaError_t unet_output_rgb(const UnetNet* n, int T, float* rgb, cudaStream_t s);
// The host's round-to-nearest-even float -> bfloat16 rule (NaN kept NaN).
void host_bf16(const float* src, size_t n, uint16_t* dst);

}  // namespace yoro
