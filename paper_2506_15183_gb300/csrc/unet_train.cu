// Training of the learned hole inpainter on the GPU: forward, loss, backward and Adam, all
// in this library's kernels.
//
// Loss of a batch: the mean over hole pixels and color channels of (s - g)^2, s the
// network's color and g the ground truth in [0, 1].  The backward pass is the chain rule
// layer by layer:
//   output layer  dz = dL/ds s (1 - s); its weight gradient and the gradient of the last
//                 activations (the 1x1 layer's transpose);
//   3x3 layer     dZ = dY where the layer's output is positive (ReLU'), rounded to
//                 bfloat16; the bias gradient sums dZ; the weight gradient correlates the
//                 layer's input with dZ over every pixel (FP32, CUDA cores: a K = pixels
//                 reduction); the input gradient is a 3x3 convolution of dZ with the
//                 kernel flipped in both directions and its channels transposed, run by the
//                 same tcgen05 kernel as the forward (no ReLU, zero bias; outputs wider than
//                 256 channels in slices);
//   routing       a concatenation splits the input gradient by channels, nearest
//                 upsampling sums each 2x2 block, 2x2 max pooling sends each window's
//                 gradient to its first maximum (row-major), and an encoder level's output
//                 gathers its skip path and its pooling path.
// Gradients of activations are FP32 (accumulated) and bfloat16 where a tensor-core
// convolution reads them.  Adam keeps FP32 master weights; after each step the forward's
// K-major bfloat16 weights and the backward's flipped, transposed ones are rebuilt.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <new>
#include <vector>

#include "unet_internal.h"
#include "yoro.h"
#include "yoro_unet.h"

namespace yoro {

namespace {

__device__ __forceinline__ float bf2f(uint16_t b) { return __uint_as_float((uint32_t)b << 16); }

__device__ __forceinline__ uint16_t f2bf(float v)
{
    const __nv_bfloat16 b = __float2bfloat16_rn(v);
    return *reinterpret_cast<const uint16_t*>(&b);
}

__device__ __forceinline__ float warp_sum(float v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__global__ void count_holes_kernel(const uint8_t* __restrict__ hole, long long n, int* __restrict__ cnt)
{
    int c = 0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        c += hole[i] != 0;
    c = (int)warp_sum((float)c);
    if ((threadIdx.x & 31) == 0 && c) atomicAdd(cnt, c);
}

// dz of the sigmoid input at every pixel (0 outside holes) and the loss.
__global__ void loss_kernel(const float* __restrict__ rgb, const uint8_t* __restrict__ gt,
                            const uint8_t* __restrict__ hole, long long npx, const int* __restrict__ cnt,
                            float* __restrict__ dzo, float* __restrict__ loss)
{
    const float inv_n = 1.0f / (3.0f * (float)max(*cnt, 1));
    float l = 0.0f;
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < npx;
         p += (long long)gridDim.x * blockDim.x) {
        const bool h = hole[p] != 0;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const float s = rgb[3 * p + c];
            const float e = s - (float)gt[3 * p + c] / 255.0f;
            dzo[3 * p + c] = h ? 2.0f * e * inv_n * s * (1.0f - s) : 0.0f;
            if (h) l += e * e;
        }
    }
    l = warp_sum(l);
    if ((threadIdx.x & 31) == 0) atomicAdd(loss, l * inv_n);
}

// Output layer backward: the gradient of d0b (added to G) and of the 1x1 weights / biases.
__global__ void out_bwd_kernel(const uint16_t* __restrict__ a, const float* __restrict__ wout,
                               const float* __restrict__ dzo, long long npx, float* __restrict__ G,
                               float* __restrict__ gw, float* __restrict__ gb)
{
    __shared__ float s[99];
    for (int i = threadIdx.x; i < 99; i += blockDim.x) s[i] = 0.0f;
    __syncthreads();
    for (long long base = blockIdx.x * (long long)blockDim.x; base < npx; base += (long long)gridDim.x * blockDim.x) {
        const long long p = base + threadIdx.x;
        float dz[3] = {0.0f, 0.0f, 0.0f};
        float av[32];
        if (p < npx) {
#pragma unroll
            for (int c = 0; c < 3; ++c) dz[c] = dzo[3 * p + c];
#pragma unroll
            for (int ci = 0; ci < 32; ++ci) av[ci] = bf2f(a[p * 32 + ci]);
#pragma unroll
            for (int ci = 0; ci < 32; ++ci)
                G[p * 32 + ci] += wout[ci] * dz[0] + wout[32 + ci] * dz[1] + wout[64 + ci] * dz[2];
        } else {
#pragma unroll
            for (int ci = 0; ci < 32; ++ci) av[ci] = 0.0f;
        }
        const bool any = __any_sync(0xffffffffu, dz[0] != 0.0f || dz[1] != 0.0f || dz[2] != 0.0f);
        if (!any) continue;  // warp-uniform: no hole pixel in this warp
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const float b = warp_sum(dz[c]);
            if ((threadIdx.x & 31) == 0) atomicAdd(&s[96 + c], b);
            for (int ci = 0; ci < 32; ++ci) {
                const float v = warp_sum(dz[c] * av[ci]);
                if ((threadIdx.x & 31) == 0) atomicAdd(&s[c * 32 + ci], v);
            }
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < 96; i += blockDim.x) atomicAdd(&gw[i], s[i]);
    for (int i = threadIdx.x; i < 3; i += blockDim.x) atomicAdd(&gb[i], s[96 + i]);
}

// dZ = G where the layer's output Y is positive (bfloat16), and the bias gradient (sum of
// dZ per channel).  Y: channel stride ycs, offset ycoff; up: Y is the 2x2-upsampled copy
// (read at (2y, 2x)) of a layer whose pixels are side x side.
__global__ void relu_mask_kernel(const float* __restrict__ G, const uint16_t* __restrict__ Y, int ycs, int ycoff,
                                 int up, int side, int C, long long n, uint16_t* __restrict__ dZ,
                                 float* __restrict__ db)
{
    __shared__ float s[256];
    for (int i = threadIdx.x; i < C; i += blockDim.x) s[i] = 0.0f;
    __syncthreads();
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
        const int c = (int)(e % C);
        const long long p = e / C;
        long long yo;
        if (!up) {
            yo = p * ycs;
        } else {
            const long long x = p % side, r = p / side, y = r % side, t = r / side;
            yo = ((t * 2 * side + 2 * y) * 2 * side + 2 * x) * ycs;
        }
        const float v = bf2f(Y[yo + ycoff + c]) > 0.0f ? G[e] : 0.0f;
        dZ[e] = f2bf(v);
        if (v != 0.0f) atomicAdd(&s[c], v);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < C; i += blockDim.x) atomicAdd(&db[i], s[i]);
}

// The weight gradient with register tiles: dW[co][ci][tap] += sum over the block's pixels
// of dZ[p][co] * X[p shifted by the tap][ci] (zero outside the tile).  A CTA takes a
// CO_T x CI_T (co, ci) tile of one tap and a range of pixels, 32 pixels per step staged in
// shared memory as floats (16-byte loads of 8 bfloat16 values; the tile side is a power
// of two, so the shift is found with shifts and masks).  Thread (tc, ti) of group g keeps
// the 4 x 4 products of co 4 tc .., ci 4 ti .. over the step's pixels g, g + G, ...
// (G = 256 / (CO_T CI_T / 16) groups), each a fused multiply-add, and adds its sums to
// dW at the end.  The channels a load covers lie inside X's channel stride (a layer whose
// input channels are padded, the first, reads the zero padding); sums for ci >= cin are
// dropped.
template <int CO_T, int CI_T>
__global__ void __launch_bounds__(256) dw_tiled_kernel(const uint16_t* __restrict__ dZ, const uint16_t* __restrict__ X,
                                                      int xcs, int side_log2, int cin, int cout, long long npx,
                                                      int pix_per_block, float* __restrict__ dW)
{
    constexpr int TC = CO_T / 4, TI = CI_T / 4, G = 256 / (TC * TI);
    __shared__ __align__(16) float sZ[32][CO_T + 4];
    __shared__ __align__(16) float sX[32][CI_T + 4];
    const int ci0 = blockIdx.x * CI_T, co0 = blockIdx.y * CO_T;
    const int tap = blockIdx.z % 9, split = blockIdx.z / 9;
    const int dy = tap / 3 - 1, dx = tap % 3 - 1;
    const int side = 1 << side_log2;
    const int t = threadIdx.x;
    const int g = t / (TC * TI), r = t - g * (TC * TI);
    const int tc = r / TI, ti = r - tc * TI;
    const long long p_begin = (long long)split * pix_per_block;
    const long long p_end = min(npx, p_begin + pix_per_block);
    float acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = 0.0f;
    for (long long p0 = p_begin; p0 < p_end; p0 += 32) {
        // dZ rows of the step: 32 pixels x CO_T channels, 8 per load
        for (int l = t; l < 32 * (CO_T / 8); l += 256) {
            const int k = l / (CO_T / 8), c = (l - k * (CO_T / 8)) * 8;
            const long long p = p0 + k;
            uint4 u = make_uint4(0u, 0u, 0u, 0u);
            if (p < p_end) u = *reinterpret_cast<const uint4*>(dZ + p * cout + co0 + c);
            float4* dst = reinterpret_cast<float4*>(&sZ[k][c]);
            dst[0] = make_float4(__uint_as_float(u.x << 16), __uint_as_float(u.x & 0xffff0000u),
                                 __uint_as_float(u.y << 16), __uint_as_float(u.y & 0xffff0000u));
            dst[1] = make_float4(__uint_as_float(u.z << 16), __uint_as_float(u.z & 0xffff0000u),
                                 __uint_as_float(u.w << 16), __uint_as_float(u.w & 0xffff0000u));
        }
        // X at the tap's shift: 32 pixels x CI_T channels
        for (int l = t; l < 32 * (CI_T / 8); l += 256) {
            const int k = l / (CI_T / 8), c = (l - k * (CI_T / 8)) * 8;
            const long long p = p0 + k;
            uint4 u = make_uint4(0u, 0u, 0u, 0u);
            if (p < p_end) {
                const int x = (int)(p & (side - 1)), y = (int)((p >> side_log2) & (side - 1));
                const long long tt = p >> (2 * side_log2);
                const int ys = y + dy, xs = x + dx;
                if (ys >= 0 && ys < side && xs >= 0 && xs < side)
                    u = *reinterpret_cast<const uint4*>(X + (((tt << side_log2) + ys) * side + xs) * xcs + ci0 + c);
            }
            float4* dst = reinterpret_cast<float4*>(&sX[k][c]);
            dst[0] = make_float4(__uint_as_float(u.x << 16), __uint_as_float(u.x & 0xffff0000u),
                                 __uint_as_float(u.y << 16), __uint_as_float(u.y & 0xffff0000u));
            dst[1] = make_float4(__uint_as_float(u.z << 16), __uint_as_float(u.z & 0xffff0000u),
                                 __uint_as_float(u.w << 16), __uint_as_float(u.w & 0xffff0000u));
        }
        __syncthreads();
#pragma unroll 4
        for (int k = g; k < 32; k += G) {
            const float4 z = *reinterpret_cast<const float4*>(&sZ[k][4 * tc]);
            const float4 x = *reinterpret_cast<const float4*>(&sX[k][4 * ti]);
            const float zv[4] = {z.x, z.y, z.z, z.w}, xv[4] = {x.x, x.y, x.z, x.w};
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = __fmaf_rn(zv[i], xv[j], acc[i][j]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int co = co0 + 4 * tc + i;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int ci = ci0 + 4 * ti + j;
            if (ci < cin) atomicAdd(&dW[((long long)co * cin + ci) * 9 + tap], acc[i][j]);
        }
    }
}

// G[p][c] += DX[p * dcs + dcoff + c]
__global__ void add_kernel(float* __restrict__ G, const uint16_t* __restrict__ DX, int dcs, int dcoff, int C,
                           long long n)
{
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x)
        G[e] += bf2f(DX[(e / C) * dcs + dcoff + e % C]);
}

// Nearest upsampling's gradient: G (side x side) += the sum of DX's 2x2 block (2 side).
__global__ void upbwd_kernel(float* __restrict__ G, const uint16_t* __restrict__ DX, int dcs, int dcoff, int side,
                             int C, long long n)
{
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
        const int c = (int)(e % C);
        const long long p = e / C, x = p % side, r = p / side, y = r % side, t = r / side;
        float s = 0.0f;
#pragma unroll
        for (int ab = 0; ab < 4; ++ab)
            s += bf2f(DX[((t * 2 * side + 2 * y + (ab >> 1)) * 2 * side + 2 * x + (ab & 1)) * dcs + dcoff + c]);
        G[e] += s;
    }
}

// 2x2 max pooling's gradient: each pooled pixel's gradient (DX, side x side, C channels)
// goes to the first maximum of its window of Y (2 side x 2 side, channel stride ycs), in
// G (2 side x 2 side x C).
__global__ void poolbwd_kernel(float* __restrict__ G, const uint16_t* __restrict__ DX, const uint16_t* __restrict__ Y,
                               int ycs, int side, int C, long long n)
{
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
        const int c = (int)(e % C);
        const long long p = e / C, x = p % side, r = p / side, y = r % side, t = r / side;
        const int s2 = 2 * side;
        long long best = -1;
        float bv = 0.0f;
#pragma unroll
        for (int ab = 0; ab < 4; ++ab) {
            const long long q = (t * s2 + 2 * y + (ab >> 1)) * s2 + 2 * x + (ab & 1);
            const float v = bf2f(Y[q * ycs + c]);
            if (best < 0 || v > bv) {
                best = q;
                bv = v;
            }
        }
        G[best * C + c] += bf2f(DX[e]);
    }
}

__global__ void adam_kernel(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m,
                            float* __restrict__ v, long long n, float lr, float b1, float b2, float eps, float c1,
                            float c2)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float mi = b1 * m[i] + (1.0f - b1) * gi;
        const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    }
}

// Forward weights: (cout, cin, 3, 3) -> K-major (cout, 9, cin_pad) bfloat16, zero padding.
__global__ void fwd_weights_kernel(const float* __restrict__ W, int cout, int cin, int cin_pad, uint16_t* __restrict__ wk)
{
    const long long n = (long long)cout * 9 * cin_pad;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const int ci = (int)(i % cin_pad);
        const long long r = i / cin_pad;
        const int tap = (int)(r % 9), co = (int)(r / 9);
        wk[i] = ci < cin ? f2bf(W[((long long)co * cin + ci) * 9 + tap]) : (uint16_t)0;
    }
}

// Backward weights: wt[ci][tap'][co] = W[co][ci][8 - tap'] (the kernel flipped in both
// directions), bfloat16: the input gradient is then a 3x3 convolution of dZ.
__global__ void bwd_weights_kernel(const float* __restrict__ W, int cout, int cin, uint16_t* __restrict__ wt)
{
    const long long n = (long long)cin * 9 * cout;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const int co = (int)(i % cout);
        const long long r = i / cout;
        const int tap = (int)(r % 9), ci = (int)(r / 9);
        wt[i] = f2bf(W[((long long)co * cin + ci) * 9 + (8 - tap)]);
    }
}

// Output layer: bfloat16-rounded weights as floats, then the FP32 biases.
__global__ void out_weights_kernel(const float* __restrict__ W, const float* __restrict__ b, float* __restrict__ wout)
{
    const int i = threadIdx.x;
    if (i < 96) wout[i] = bf2f(f2bf(W[i]));
    if (i < 3) wout[96 + i] = b[i];
}

int blocks_for(long long n, int per = 256) { return (int)std::min<long long>((n + per - 1) / per, 8192); }

}  // namespace

struct Trainer {
    UnetNet* net;
    int B;
    size_t np;
    float *params, *grads, *m, *v;
    size_t woff[14], boff[14], wout_off, bout_off;
    uint16_t* wt[14];
    float* G[14];
    uint16_t *dZ, *DX;
    float *zero_bias, *rgb, *dzo, *loss;
    int* nhole;
    int step;
    float lr, b1, b2, eps;
};

namespace {

int layer_side(int i) { return i < 8 ? (64 >> (i / 2)) : (64 >> (2 - (i - 8) / 2)); }

void trainer_free(Trainer* t)
{
    if (!t) return;
    unet_free(t->net);
    for (int i = 0; i < 14; ++i) {
        cudaFree(t->wt[i]);
        cudaFree(t->G[i]);
    }
    void* bufs[] = {t->params, t->grads, t->m, t->v, t->dZ, t->DX, t->zero_bias, t->rgb, t->dzo, t->loss, t->nhole};
    for (void* b : bufs) cudaFree(b);
    delete t;
}

cudaError_t rebuild_weights(Trainer* t, cudaStream_t s)
{
    UnetNet* n = t->net;
    for (int i = 0; i < 14; ++i) {
        const UnetLayer& L = n->conv[i];
        const float* W = t->params + t->woff[i];
        fwd_weights_kernel<<<blocks_for((long long)L.cout * 9 * L.cin_pad), 256, 0, s>>>(W, L.cout, L.cin, L.cin_pad,
                                                                                       L.wk);
        bwd_weights_kernel<<<blocks_for((long long)L.cin * 9 * L.cout), 256, 0, s>>>(W, L.cout, L.cin, t->wt[i]);
        const cudaError_t e = cudaMemcpyAsync(L.bias, t->params + t->boff[i], L.cout * 4, cudaMemcpyDeviceToDevice, s);
        if (e != cudaSuccess) return e;
    }
    out_weights_kernel<<<1, 128, 0, s>>>(t->params + t->wout_off, t->params + t->bout_off, n->wout);
    return cudaGetLastError();
}

}  // namespace

Trainer* trainer_create(const float* params, size_t np, int batch, float lr, float b1, float b2, float eps)
{
    if (!params || np != unet_param_count() || batch < 2 || (batch & 1)) return nullptr;
    Trainer* t = new (std::nothrow) Trainer();
    if (!t) return nullptr;
    std::memset(t, 0, sizeof *t);
    t->B = batch;
    t->np = np;
    t->lr = lr;
    t->b1 = b1;
    t->b2 = b2;
    t->eps = eps;
    t->net = unet_create(params, np, batch, 1);
    bool ok = t->net != nullptr;
    size_t off = 0;
    for (int i = 0; i < 14; ++i) {
        int cin, cout;
        unet_layer_dims(i, &cin, &cout);
        t->woff[i] = off;
        off += (size_t)cout * cin * 9;
        t->boff[i] = off;
        off += cout;
    }
    t->wout_off = off;
    t->bout_off = off + 96;
    const size_t B = batch;
    size_t dz_max = 0, dx_max = 0;
    for (int i = 0; i < 14 && ok; ++i) {
        int cin, cout;
        unet_layer_dims(i, &cin, &cout);
        const size_t P = B * layer_side(i) * layer_side(i);
        dz_max = std::max(dz_max, P * cout);
        dx_max = std::max(dx_max, P * (size_t)((cin + 31) / 32 * 32));
        ok = cudaMalloc(&t->wt[i], (size_t)cin * 9 * cout * 2) == cudaSuccess &&
             cudaMalloc(&t->G[i], P * cout * 4) == cudaSuccess;
    }
    if (ok)
        ok = cudaMalloc(&t->params, np * 4) == cudaSuccess && cudaMalloc(&t->grads, np * 4) == cudaSuccess &&
             cudaMalloc(&t->m, np * 4) == cudaSuccess && cudaMalloc(&t->v, np * 4) == cudaSuccess &&
             cudaMalloc(&t->dZ, dz_max * 2) == cudaSuccess && cudaMalloc(&t->DX, dx_max * 2) == cudaSuccess &&
             cudaMalloc(&t->zero_bias, 384 * 4) == cudaSuccess && cudaMalloc(&t->rgb, B * 4096 * 3 * 4) == cudaSuccess &&
             cudaMalloc(&t->dzo, B * 4096 * 3 * 4) == cudaSuccess && cudaMalloc(&t->loss, 4) == cudaSuccess &&
             cudaMalloc(&t->nhole, 4) == cudaSuccess;
    if (ok)
        ok = cudaMemcpy(t->params, params, np * 4, cudaMemcpyHostToDevice) == cudaSuccess &&
             cudaMemset(t->m, 0, np * 4) == cudaSuccess && cudaMemset(t->v, 0, np * 4) == cudaSuccess &&
             cudaMemset(t->zero_bias, 0, 384 * 4) == cudaSuccess && cudaMemset(t->grads, 0, np * 4) == cudaSuccess &&
             rebuild_weights(t, nullptr) == cudaSuccess && cudaDeviceSynchronize() == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        trainer_free(t);
        return nullptr;
    }
    return t;
}

// One step on B tiles (B even, <= the trainer's batch): x (B x 64 x 64 x 32 bfloat16), gt
// (B x 64 x 64 x 3 bytes), hole (B x 64 x 64 bytes).  lr = 0 leaves the weights as they
// are (the gradients stay readable).
cudaError_t trainer_step(Trainer* t, const void* x, const uint8_t* gt, const uint8_t* hole, int B, cudaStream_t s)
{
    UnetNet* n = t->net;
    const long long npx = (long long)B * 4096;
    cudaError_t e = cudaMemsetAsync(t->grads, 0, t->np * 4, s);
    for (int i = 0; i < 14 && e == cudaSuccess; ++i) {
        int cin, cout;
        unet_layer_dims(i, &cin, &cout);
        e = cudaMemsetAsync(t->G[i], 0, (size_t)B * layer_side(i) * layer_side(i) * cout * 4, s);
    }
    if (e == cudaSuccess) e = cudaMemsetAsync(t->loss, 0, 4, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(t->nhole, 0, 4, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(n->in0, x, (size_t)npx * 32 * 2, cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess) e = unet_run(n, B, nullptr, s);
    if (e == cudaSuccess) e = unet_output_rgb(n, B, t->rgb, s);
    if (e != cudaSuccess) return e;
    count_holes_kernel<<<blocks_for(npx), 256, 0, s>>>(hole, npx, t->nhole);
    loss_kernel<<<blocks_for(npx), 256, 0, s>>>(t->rgb, gt, hole, npx, t->nhole, t->dzo, t->loss);
    out_bwd_kernel<<<blocks_for(npx), 256, 0, s>>>(n->d0b, n->wout, t->dzo, npx, t->G[13], t->grads + t->wout_off,
                                                  t->grads + t->bout_off);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;

    // per layer: forward input X (channel stride), output Y (stride, offset, upsampled copy)
    struct IO {
        const uint16_t* x;
        int xcs;
        const uint16_t* y;
        int ycs, ycoff, yup;
    };
    const IO io[14] = {{n->in0, 32, n->e0a, 32, 0, 0},   {n->e0a, 32, n->cat0, 96, 0, 0},
                       {n->p0, 32, n->e1a, 64, 0, 0},    {n->e1a, 64, n->cat1, 192, 0, 0},
                       {n->p1, 64, n->e2a, 128, 0, 0},   {n->e2a, 128, n->cat2, 384, 0, 0},
                       {n->p2, 128, n->e3a, 256, 0, 0},  {n->e3a, 256, n->cat2, 384, 128, 1},
                       {n->cat2, 384, n->d2a, 128, 0, 0}, {n->d2a, 128, n->cat1, 192, 64, 1},
                       {n->cat1, 192, n->d1a, 64, 0, 0}, {n->d1a, 64, n->cat0, 96, 32, 1},
                       {n->cat0, 96, n->d0a, 32, 0, 0},  {n->d0a, 32, n->d0b, 32, 0, 0}};
    for (int i = 13; i >= 0; --i) {
        const UnetLayer& L = n->conv[i];
        const int side = layer_side(i);
        const long long P = (long long)B * side * side;
        const long long nz = P * L.cout;
        relu_mask_kernel<<<blocks_for(nz), 256, 0, s>>>(t->G[i], io[i].y, io[i].ycs, io[i].ycoff, io[i].yup, side,
                                                        L.cout, nz, t->dZ, t->grads + t->boff[i]);
        {
            // (co, ci) tiles of 64 where the channels allow, else 32; pixel ranges (multiples
            // of 32) short enough for at least ~1,000 CTAs
            const int cot = L.cout % 64 == 0 ? 64 : 32, cit = L.cin % 64 == 0 ? 64 : 32;
            const int tiles = (L.cin + cit - 1) / cit * (L.cout / cot) * 9;
            long long ppb = 4096;
            while (ppb > 256 && tiles * ((P + ppb - 1) / ppb) < 1024) ppb /= 2;
            const dim3 grid((L.cin + cit - 1) / cit, L.cout / cot, (unsigned)(9 * ((P + ppb - 1) / ppb)));
            int ls = 0;
            while ((1 << ls) < side) ++ls;
            float* dw = t->grads + t->woff[i];
            if (cot == 64 && cit == 64)
                dw_tiled_kernel<64, 64><<<grid, 256, 0, s>>>(t->dZ, io[i].x, io[i].xcs, ls, L.cin, L.cout, P, (int)ppb, dw);
            else if (cot == 64)
                dw_tiled_kernel<64, 32><<<grid, 256, 0, s>>>(t->dZ, io[i].x, io[i].xcs, ls, L.cin, L.cout, P, (int)ppb, dw);
            else if (cit == 64)
                dw_tiled_kernel<32, 64><<<grid, 256, 0, s>>>(t->dZ, io[i].x, io[i].xcs, ls, L.cin, L.cout, P, (int)ppb, dw);
            else
                dw_tiled_kernel<32, 32><<<grid, 256, 0, s>>>(t->dZ, io[i].x, io[i].xcs, ls, L.cin, L.cout, P, (int)ppb, dw);
        }
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        if (i == 0) break;
        // input gradient: slices of 256 / 128 / 64 / 32 output channels
        for (int c0 = 0; c0 < L.cin && e == cudaSuccess;) {
            const int rem = L.cin - c0;
            const int w = rem >= 256 ? 256 : rem >= 128 ? 128 : rem >= 64 ? 64 : 32;
            e = unet_conv3x3(t->dZ, B, side, side, L.cout, t->wt[i] + (size_t)c0 * 9 * L.cout, t->zero_bias, t->DX,
                             w, L.cin, c0, 0, 0, s);
            c0 += w;
        }
        if (e != cudaSuccess) return e;
        // route the input gradient to the producers' output gradients
        auto add = [&](int dst, int coff, int C) {
            const long long nn = P * C;
            add_kernel<<<blocks_for(nn), 256, 0, s>>>(t->G[dst], t->DX, L.cin, coff, C, nn);
        };
        auto upb = [&](int dst, int coff, int C) {
            const long long nn = P / 4 * C;
            upbwd_kernel<<<blocks_for(nn), 256, 0, s>>>(t->G[dst], t->DX, L.cin, coff, side / 2, C, nn);
        };
        auto pool = [&](int dst, const uint16_t* y, int ycs) {
            const long long nn = P * L.cin;
            poolbwd_kernel<<<blocks_for(nn), 256, 0, s>>>(t->G[dst], t->DX, y, ycs, side, L.cin, nn);
        };
        switch (i) {
            case 13: add(12, 0, 32); break;
            case 12: add(1, 0, 32); upb(11, 32, 64); break;
            case 11: add(10, 0, 64); break;
            case 10: add(3, 0, 64); upb(9, 64, 128); break;
            case 9: add(8, 0, 128); break;
            case 8: add(5, 0, 128); upb(7, 128, 256); break;
            case 7: add(6, 0, 256); break;
            case 6: pool(5, n->cat2, 384); break;
            case 5: add(4, 0, 128); break;
            case 4: pool(3, n->cat1, 192); break;
            case 3: add(2, 0, 64); break;
            case 2: pool(1, n->cat0, 96); break;
            case 1: add(0, 0, 32); break;
        }
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    if (t->lr != 0.0f) {
        ++t->step;
        const float c1 = 1.0f - std::pow(t->b1, (float)t->step), c2 = 1.0f - std::pow(t->b2, (float)t->step);
        adam_kernel<<<blocks_for((long long)t->np), 256, 0, s>>>(t->params, t->grads, t->m, t->v, (long long)t->np,
                                                                t->lr, t->b1, t->b2, t->eps, c1, c2);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        e = rebuild_weights(t, s);
    }
    return e;
}

}  // namespace yoro

struct yoro_unet_trainer_ctx {
    yoro::Trainer* t;
};

extern "C" {

yoro_unet_trainer yoro_unet_trainer_create(const float* params, long long n_params, int batch_tiles, float lr,
                                           float beta1, float beta2, float eps)
{
    if (!params || n_params <= 0 || !(lr >= 0.0f) || !(beta1 >= 0.0f && beta1 < 1.0f) ||
        !(beta2 >= 0.0f && beta2 < 1.0f) || !(eps > 0.0f))
        return nullptr;
    yoro::Trainer* t = yoro::trainer_create(params, (size_t)n_params, batch_tiles, lr, beta1, beta2, eps);
    if (!t) return nullptr;
    yoro_unet_trainer_ctx* c = new (std::nothrow) yoro_unet_trainer_ctx();
    if (!c) {
        yoro::trainer_free(t);
        return nullptr;
    }
    c->t = t;
    return c;
}

void yoro_unet_trainer_destroy(yoro_unet_trainer tr)
{
    if (!tr) return;
    yoro::trainer_free(tr->t);
    delete tr;
}

yoro_status yoro_unet_train_step(yoro_unet_trainer tr, const void* x, const unsigned char* gt,
                                 const unsigned char* hole, int tiles, void* cuda_stream)
{
    if (!tr || !x || !gt || !hole || tiles < 2 || (tiles & 1) || tiles > tr->t->B) return YORO_EINVAL;
    if ((uintptr_t)x & 15u) return YORO_EALIGN;
    return yoro::trainer_step(tr->t, x, gt, hole, tiles, (cudaStream_t)cuda_stream) == cudaSuccess ? YORO_OK
                                                                                                 : YORO_ECUDA;
}

yoro_status yoro_unet_trainer_set_lr(yoro_unet_trainer tr, float lr)
{
    if (!tr || !(lr >= 0.0f) || !std::isfinite(lr)) return YORO_EINVAL;
    tr->t->lr = lr;
    return YORO_OK;
}

yoro_status yoro_unet_trainer_read(yoro_unet_trainer tr, int what, float* host_out, void* cuda_stream)
{
    if (!tr || !host_out || what < 0 || what > 2) return YORO_EINVAL;
    const cudaStream_t s = (cudaStream_t)cuda_stream;
    const float* src = what == 0 ? tr->t->params : what == 1 ? tr->t->grads : tr->t->loss;
    const size_t bytes = what == 2 ? 4 : tr->t->np * 4;
    if (cudaMemcpyAsync(host_out, src, bytes, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess) {
        cudaGetLastError();
        return YORO_ECUDA;
    }
    return YORO_OK;
}

}  // extern "C"
