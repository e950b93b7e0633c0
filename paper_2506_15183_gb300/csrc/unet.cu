// The learned hole inpainter on the tensor cores (sm_103a): a 4-level U-Net over
// 64 x 64 tiles, BF16 weights and activations, FP32 accumulation.
//
// Each 3x3 convolution is an implicit GEMM: M = output pixels (128 per CTA tile, whole
// rows of one or two tiles), N = output channels (32..256, one MMA tile), K = 9 taps x
// input channels, taken 32 channels of one tap at a time.  A K step is two TMA tiled
// loads into shared memory with 64-byte swizzle: the activation box {32 channels, W, Hb,
// Nb} of NHWC bf16 at the tap's offset (the padding rows and columns are outside the
// tensor and arrive as zeros), and the weight box {32, Cout} of the K-major weights
// (k = tap * Cin + ci).  One thread issues the copies, another the tcgen05.mma (kind::f16,
// BF16 operands, FP32 accumulator in tensor memory, two K = 16 steps per stage), with
// mbarriers between them (4 stages).  The epilogue reads the accumulators with
// tcgen05.ld, adds the bias, applies ReLU, rounds to BF16 and stores NHWC at a channel
// offset of a wider buffer (so a decoder's concatenation is written in place), or, for
// the layer below a decoder level, to the 2 x 2 pixels of the nearest upsampling.
//
// Every wait on an mbarrier has a deadline (1 s of %globaltimer): a wait that runs out
// records kUnetTimeout in a status word, the kernel waits (again bounded) for the copies
// it issued, frees its tensor memory and returns.  Nothing traps.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>
#include <cstring>

#include "yoro.h"
#include "yoro_internal.h"
#include "yoro_unet.h"

namespace yoro {

namespace {

__device__ unsigned g_unet_status;  // kernel-side failures of this file's kernels

constexpr unsigned kUnetTimeout = 1u;
constexpr int kStages = 4;
constexpr int kTileM = 128;                  // pixels per CTA tile (MMA M)
constexpr int kKc = 32;                      // channels per K step (64 bytes: the swizzle span)
constexpr int kABytes = kTileM * kKc * 2;    // 8 KB
constexpr uint64_t kWaitNs = 1000000000ull;  // 1 s

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ uint64_t globaltimer()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Wait for the phase of parity `parity` to complete; false if `deadline` passed first.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, uint64_t deadline)
{
    while (!mbar_try_wait(bar, parity))
        if (globaltimer() > deadline) return false;
    return true;
}

__device__ __forceinline__ void tma_load_4d(void* dst, const CUtensorMap* map, uint64_t* bar, int c0, int c1, int c2,
                                            int c3)
{
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4, %5, %6}], "
        "[%2];" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(smem_u32(bar)), "r"(c0), "r"(c1), "r"(c2), "r"(c3)
        : "memory");
}

__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, uint64_t* bar, int c0, int c1)
{
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4}], [%2];" ::"r"(
            smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(smem_u32(bar)), "r"(c0), "r"(c1)
        : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// Shared-memory matrix descriptor of a K-major operand whose rows (one M or N index
// each) are 64 bytes of K, 64-byte swizzled by the copy engine: 8-row groups 512 bytes
// apart (stride byte offset), leading byte offset unused for a swizzled K-major layout,
// descriptor version 1, layout type 4 (64-byte swizzle).  The start address may move
// by 32 bytes inside the swizzle span to select the second K = 16 half.
__device__ __forceinline__ uint64_t desc_sw64(uint32_t saddr)
{
    uint64_t d = (uint64_t)((saddr >> 4) & 0x3fffu);
    d |= (uint64_t)1u << 16;
    d |= (uint64_t)(512u >> 4) << 32;
    d |= (uint64_t)1u << 46;
    d |= (uint64_t)4u << 61;
    return d;
}

// Instruction descriptor of kind::f16: FP32 accumulator (bits 4-5 = 1), BF16 A and B
// (bits 7-9 and 10-12 = 1), both K-major, N / 8 at bit 17, M / 16 at bit 24.
__device__ __forceinline__ uint32_t idesc_bf16(int n)
{
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(kTileM >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t accum)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(idesc), "r"(accum)
        : "memory");
}

__device__ __forceinline__ void mma_commit(uint64_t* bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}

// 32 consecutive accumulator columns of this warp's 32 TMEM lanes (one lane per thread).
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&r)[32])
{
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ uint32_t pack_bf16x2(float lo, float hi)
{
    const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<const uint32_t*>(&v);
}

struct ConvArgs {
    int T, H, W;          // tiles and their size (the output has the input's size)
    int Cin, Cout;        // Cin: channels of the input tensor, a multiple of 32
    const float* bias;    // Cout
    __nv_bfloat16* y;     // NHWC output, channel stride y_cstride, channels from y_coff
    int y_cstride, y_coff;
    int upsample;         // 1: pixel (yy, xx) goes to (2yy + a, 2xx + b), a, b in {0, 1}
    int relu;
    int ncols;            // tensor-memory columns allocated (a power of two >= Cout, >= 32)
};

__global__ void __launch_bounds__(128, 1)
    conv3x3_tc(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, const ConvArgs a)
{
    extern __shared__ unsigned char smem_raw[];
    unsigned char* smem = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) &
                                                           ~static_cast<uintptr_t>(1023));
    const int b_bytes = a.Cout * kKc * 2;
    const int stage_bytes = kABytes + ((b_bytes + 1023) & ~1023);
    uint64_t* full = reinterpret_cast<uint64_t*>(smem + kStages * stage_bytes);
    uint64_t* empty = full + kStages;
    uint64_t* done = empty + kStages;
    uint32_t* tslot = reinterpret_cast<uint32_t*>(done + 1);
    volatile int* counts = reinterpret_cast<volatile int*>(tslot + 1);  // [0] issued, [1] consumed
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

    if (threadIdx.x == 0) {
        for (int s = 0; s < kStages; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        mbar_init(done, 1);
        counts[0] = 0;
        counts[1] = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tslot)),
                     "r"(a.ncols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tslot;

    const int cb_n = a.Cin / kKc;
    const int nk = 9 * cb_n;
    const int hw = a.H * a.W;
    const int p0 = blockIdx.x * kTileM;
    const int n0 = p0 / hw;
    const int y0 = (p0 - n0 * hw) / a.W;
    const uint64_t deadline = globaltimer() + kWaitNs;

    if (warp == 0 && lane == 0) {  // copies
        int k = 0;
        for (; k < nk; ++k) {
            const int s = k % kStages;
            if (!mbar_wait(&empty[s], ((k / kStages) & 1) ^ 1, deadline)) {
                atomicOr(&g_unet_status, kUnetTimeout);
                break;
            }
            const int tap = k / cb_n, cb = k - tap * cb_n;
            const int dy = tap / 3, dx = tap - 3 * (tap / 3);
            unsigned char* sa = smem + s * stage_bytes;
            mbar_expect_tx(&full[s], (uint32_t)(kABytes + b_bytes));
            tma_load_4d(sa, &tmA, &full[s], cb * kKc, dx - 1, y0 + dy - 1, n0);
            tma_load_2d(sa + kABytes, &tmB, &full[s], tap * a.Cin + cb * kKc, 0);
            counts[0] = k + 1;
        }
    } else if (warp == 1 && lane == 0) {  // MMAs
        const uint32_t idesc = idesc_bf16(a.Cout);
        for (int k = 0; k < nk; ++k) {
            const int s = k % kStages;
            if (!mbar_wait(&full[s], (k / kStages) & 1, deadline)) {
                atomicOr(&g_unet_status, kUnetTimeout);
                break;
            }
            tc_fence_after();
            const uint32_t sa = smem_u32(smem + s * stage_bytes), sb = sa + kABytes;
            mma_bf16(tmem, desc_sw64(sa), desc_sw64(sb), idesc, k > 0 ? 1u : 0u);
            mma_bf16(tmem, desc_sw64(sa + 32), desc_sw64(sb + 32), idesc, 1u);
            mma_commit(&empty[s]);
            counts[1] = k + 1;
        }
        mma_commit(done);  // arrives once every MMA issued above has completed
    }
    __syncwarp();

    const bool ok = mbar_wait(done, 0, deadline + kWaitNs);
    if (!ok) atomicOr(&g_unet_status, kUnetTimeout);
    if (ok) {
        tc_fence_after();
        const int m = warp * 32 + lane;  // this thread's pixel of the tile = its TMEM lane
        const int p = p0 + m;
        const int n = p / hw, rem = p - n * hw, yy = rem / a.W, xx = rem - (rem / a.W) * a.W;
        for (int c0 = 0; c0 < a.Cout; c0 += 32) {
            uint32_t r[32];
            tmem_ld32(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, r);
            uint4 q[4];
            uint32_t* qw = reinterpret_cast<uint32_t*>(q);
#pragma unroll
            for (int i = 0; i < 16; ++i) {
                float v0 = __fadd_rn(__uint_as_float(r[2 * i]), __ldg(a.bias + c0 + 2 * i));
                float v1 = __fadd_rn(__uint_as_float(r[2 * i + 1]), __ldg(a.bias + c0 + 2 * i + 1));
                if (a.relu) {
                    v0 = fmaxf(v0, 0.0f);
                    v1 = fmaxf(v1, 0.0f);
                }
                qw[i] = pack_bf16x2(v0, v1);
            }
            if (!a.upsample) {
                uint4* dst = reinterpret_cast<uint4*>(a.y + ((size_t)p * a.y_cstride + a.y_coff + c0));
#pragma unroll
                for (int i = 0; i < 4; ++i) dst[i] = q[i];
            } else {
                const int W2 = 2 * a.W, H2 = 2 * a.H;
#pragma unroll
                for (int ab = 0; ab < 4; ++ab) {
                    const size_t op = ((size_t)n * H2 + (2 * yy + (ab >> 1))) * W2 + (2 * xx + (ab & 1));
                    uint4* dst = reinterpret_cast<uint4*>(a.y + (op * a.y_cstride + a.y_coff + c0));
#pragma unroll
                    for (int i = 0; i < 4; ++i) dst[i] = q[i];
                }
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (threadIdx.x == 0) {  // copies still in flight after a timeout: wait for them (bounded)
        const uint64_t d2 = globaltimer() + kWaitNs;
        for (int k = counts[1]; k < counts[0]; ++k)
            if (!mbar_wait(&full[k % kStages], (k / kStages) & 1, d2)) break;
    }
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(a.ncols) : "memory");
    }
}

// Driver entry point for tensor-map encoding, looked up once through the runtime (no
// link against the driver library).
using EncodeTiled = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                 const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                 CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiled encode_fn()
{
    static EncodeTiled fn = nullptr;
    if (!fn) {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) !=
                cudaSuccess ||
            q != cudaDriverEntryPointSuccess)
            return nullptr;
        fn = reinterpret_cast<EncodeTiled>(p);
    }
    return fn;
}

size_t conv_smem_bytes(int cout)
{
    const int b_bytes = cout * kKc * 2;
    const int stage = kABytes + ((b_bytes + 1023) & ~1023);
    return 1024 + (size_t)kStages * stage + (2 * kStages + 1) * 8 + 16;
}

}  // namespace

unsigned unet_status_take()
{
    unsigned v = 0, z = 0;
    if (cudaMemcpyFromSymbol(&v, g_unet_status, sizeof v) != cudaSuccess ||
        cudaMemcpyToSymbol(g_unet_status, &z, sizeof z) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return v;
}

// One 3x3 convolution (zero padding 1) of x (T tiles of H x W, NHWC bf16 with Cin
// channels, Cin a multiple of 32) with K-major weights wk (Cout rows of 9 Cin, k = (3 dy +
// dx) Cin + ci) and bias, ReLU if relu, into y at channel offset y_coff of a tensor with
// y_cstride channels (upsample: into the 2H x 2W grid of the nearest upsampling).
// Needs T H W a multiple of 128, W in {8, 16, 32, 64, 128} with 128 / W rows per tile or
// whole tiles per 128 pixels, Cout in {32, 64, 128, 256}.  Returns cudaErrorInvalidValue
// for shapes it does not take.
cudaError_t unet_conv3x3(const void* x, int T, int H, int W, int Cin, const void* wk, const float* bias, void* y,
                         int Cout, int y_cstride, int y_coff, int upsample, int relu, cudaStream_t stream)
{
    if (T < 1 || H < 1 || W < 1 || Cin < kKc || Cin % kKc || (Cout != 32 && Cout != 64 && Cout != 128 && Cout != 256))
        return cudaErrorInvalidValue;
    if (W > kTileM || kTileM % W) return cudaErrorInvalidValue;
    int hb = kTileM / W, nb = 1;
    if (hb > H) {
        if (hb % H) return cudaErrorInvalidValue;
        nb = hb / H;
        hb = H;
    } else if (H % hb) {
        return cudaErrorInvalidValue;
    }
    const long long pixels = (long long)T * H * W;
    if (pixels % kTileM || (nb > 1 && T % nb)) return cudaErrorInvalidValue;
    if (y_cstride % 8 || y_coff % 8 || y_coff + Cout > y_cstride) return cudaErrorInvalidValue;
    EncodeTiled enc = encode_fn();
    if (!enc) return cudaErrorNotSupported;

    CUtensorMap ta, tb;
    const cuuint64_t adim[4] = {(cuuint64_t)Cin, (cuuint64_t)W, (cuuint64_t)H, (cuuint64_t)T};
    const cuuint64_t astr[3] = {(cuuint64_t)Cin * 2, (cuuint64_t)W * Cin * 2, (cuuint64_t)H * W * Cin * 2};
    const cuuint32_t abox[4] = {(cuuint32_t)kKc, (cuuint32_t)W, (cuuint32_t)hb, (cuuint32_t)nb};
    const cuuint32_t one4[4] = {1, 1, 1, 1};
    if (enc(&ta, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, const_cast<void*>(x), adim, astr, abox, one4,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
        return cudaErrorInvalidValue;
    const cuuint64_t bdim[2] = {(cuuint64_t)9 * Cin, (cuuint64_t)Cout};
    const cuuint64_t bstr[1] = {(cuuint64_t)9 * Cin * 2};
    const cuuint32_t bbox[2] = {(cuuint32_t)kKc, (cuuint32_t)Cout};
    if (enc(&tb, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(wk), bdim, bstr, bbox, one4,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
        return cudaErrorInvalidValue;

    ConvArgs a;
    a.T = T;
    a.H = H;
    a.W = W;
    a.Cin = Cin;
    a.Cout = Cout;
    a.bias = bias;
    a.y = static_cast<__nv_bfloat16*>(y);
    a.y_cstride = y_cstride;
    a.y_coff = y_coff;
    a.upsample = upsample;
    a.relu = relu;
    a.ncols = Cout < 32 ? 32 : Cout;
    const size_t smem = conv_smem_bytes(Cout);
    static bool configured = false;
    if (!configured) {
        const cudaError_t e =
            cudaFuncSetAttribute(conv3x3_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)conv_smem_bytes(256));
        if (e != cudaSuccess) return e;
        configured = true;
    }
    conv3x3_tc<<<(unsigned)(pixels / kTileM), 128, smem, stream>>>(ta, tb, a);
    return cudaGetLastError();
}

}  // namespace yoro

extern "C" {

yoro_status yoro_unet_conv3x3(const void* x, int T, int H, int W, int Cin, const void* wk, const float* bias,
                              void* y, int Cout, int y_cstride, int y_coff, int upsample, int relu,
                              void* cuda_stream)
{
    if (!x || !wk || !bias || !y) return YORO_EINVAL;
    if (((uintptr_t)x | (uintptr_t)wk | (uintptr_t)y) & 15u) return YORO_EALIGN;
    const cudaError_t e = yoro::unet_conv3x3(x, T, H, W, Cin, wk, bias, y, Cout, y_cstride, y_coff, upsample, relu,
                                             (cudaStream_t)cuda_stream);
    if (e == cudaErrorInvalidValue) return YORO_EINVAL;
    return e == cudaSuccess ? YORO_OK : YORO_ECUDA;
}

yoro_status yoro_unet_status(void* cuda_stream)
{
    if (cudaStreamSynchronize((cudaStream_t)cuda_stream) != cudaSuccess) {
        cudaGetLastError();
        return YORO_ECUDA;
    }
    return yoro::unet_status_take() ? YORO_EDEVICE : YORO_OK;
}

}  // extern "C"
