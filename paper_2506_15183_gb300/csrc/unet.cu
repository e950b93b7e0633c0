// The learned hole inpainter on the tensor cores (sm_103a): a 4-level U-Net over
// 64 x 64 tiles, BF16 weights and activations, FP32 accumulation.
//
// Each 3x3 convolution is an implicit GEMM: M = output pixels (128 per accumulator), N =
// output channels (32..256, one MMA tile), K = taps x input channels, taken 32 channels
// (64 bytes: the swizzle span) at a time.  Operands are TMA tiled loads into shared
// memory with 64-byte swizzle (the zero padding of the convolution is the part of a box
// outside the tensor, which TMA fills with zeros); one thread issues the copies, another
// the tcgen05.mma (kind::f16, BF16 operands, FP32 accumulator in tensor memory, two
// K = 16 steps per 32-channel slice), with mbarriers between them.  The epilogue reads
// the accumulators with tcgen05.ld, adds the bias, applies ReLU, rounds to BF16 and
// stores NHWC at a channel offset of a wider buffer (so a decoder's concatenation is
// written in place), or, for the layer below a decoder level, to the 2 x 2 pixels of the
// nearest upsampling.  Two forms:
//   - conv3x3_halo, for tiles of whole rows of one image: a band of 256 / W rows goes
//     into two accumulators (each CTA walks bands blockIdx.x, + gridDim.x, ..., as many
//     CTAs as fit on the SMs at once); a K step is one (channel block, dx) pair, a single box of
//     the rows plus one above and below, shared by the three dy taps through the start
//     address of the MMA operand (whole 512-byte swizzle atoms apart), and the three
//     taps' weight boxes.  Each input pixel is copied 3 (R + 2) / R times instead of 9.
//   - conv3x3_tc, one CTA per 128-pixel tile (the 8 x 8 level, where 128 pixels are two
//     tiles, and 256 output channels): a K step is one (channel block, tap), the
//     activation box {32 channels, W, rows, tiles} at the tap's offset and the weight box
//     {32, Cout} of the K-major weights (k = tap * Cin + ci), in a 4-stage ring.
// Both use CTAs of 128 threads, several per SM, so the copies of one overlap the set-up,
// MMAs and epilogue of the others.
//
// Every wait on an mbarrier has a deadline (1 s of %globaltimer): a wait that runs out
// records kUnetTimeout in a status word, the kernel waits (again bounded) for the copies
// it issued, frees its tensor memory and returns.  Nothing traps.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <new>
#include <vector>

#include "yoro.h"
#include "yoro_internal.h"
#include "yoro_unet.h"
#include "unet_internal.h"

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

// TMA tensor stores from shared memory (bulk-group completion): 4-D and 5-D boxes.
__device__ __forceinline__ void tma_store_4d(const CUtensorMap* map, const void* src, int c0, int c1, int c2, int c3)
{
    asm volatile("cp.async.bulk.tensor.4d.global.shared::cta.bulk_group [%0, {%2, %3, %4, %5}], [%1];" ::"l"(
                     reinterpret_cast<uint64_t>(map)),
                 "r"(smem_u32(src)), "r"(c0), "r"(c1), "r"(c2), "r"(c3)
                 : "memory");
}

__device__ __forceinline__ void tma_store_5d(const CUtensorMap* map, const void* src, int c0, int c1, int c2, int c3,
                                             int c4)
{
    asm volatile("cp.async.bulk.tensor.5d.global.shared::cta.bulk_group [%0, {%2, %3, %4, %5, %6}], [%1];" ::"l"(
                     reinterpret_cast<uint64_t>(map)),
                 "r"(smem_u32(src)), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(c4)
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
    int ncols;            // tensor-memory columns allocated (a power of two >= mt Cout, >= 32)
    const int* count;     // optional: tiles at or after *count are skipped (the tile list's length)
    int mt, stages;       // halo form: 128-pixel accumulators per CTA and copy stages
};

// The epilogue of both forms: the CTA's mt accumulators of 128 pixels (pixel i of
// accumulator j is the CTA tile's pixel 128 j + i, row-major over its rows) are read
// back 32 channels at a time, the bias added, ReLU applied, rounded to BF16 and staged in
// shared memory (`stg`, 1024-aligned: the copy stages, free once every MMA has
// completed), one slice of 64 bytes per pixel for each 32 channels, in the 64-byte
// swizzle (16-byte chunk k of pixel p at p 64 + (k ^ (p / 2 mod 4)) 16, so a warp's
// writes meet no bank twice).  One thread then writes every slice with TMA tensor
// stores: a box {32 channels, W, rows, images} at channel y_coff + 32 s, or, for the
// nearest upsampling, the same box four times through a 5-D view of the output that
// splits each coordinate into (pixel, replica).  The CTA ends once the stores have read
// shared memory.
__device__ __forceinline__ void epilogue_store(const ConvArgs& a, const CUtensorMap* tmY, uint32_t tmem,
                                               unsigned char* stg, const float* bias, int mt, int n0, int y0)
{
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int m = warp * 32 + lane;  // this thread's pixel of each accumulator = its TMEM lane
    const int slice = mt * kTileM * 64;
    for (int c0 = 0; c0 < a.Cout; c0 += 32) {
        unsigned char* sl = stg + (c0 >> 5) * slice;
        for (int j = 0; j < mt; ++j) {
            uint32_t r[32];
            tmem_ld32(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(j * a.Cout + c0), r);
            uint4 q[4];
            uint32_t* qw = reinterpret_cast<uint32_t*>(q);
#pragma unroll
            for (int i = 0; i < 16; ++i) {
                float v0 = __fadd_rn(__uint_as_float(r[2 * i]), bias[c0 + 2 * i]);
                float v1 = __fadd_rn(__uint_as_float(r[2 * i + 1]), bias[c0 + 2 * i + 1]);
                if (a.relu) {
                    v0 = fmaxf(v0, 0.0f);
                    v1 = fmaxf(v1, 0.0f);
                }
                qw[i] = pack_bf16x2(v0, v1);
            }
            const int px = j * kTileM + m;
            unsigned char* row = sl + px * 64;
            const int sw = (px >> 1) & 3;
#pragma unroll
            for (int k = 0; k < 4; ++k) *reinterpret_cast<uint4*>(row + ((k ^ sw) << 4)) = q[k];
        }
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // the writes, seen by the copy engine
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int c0 = 0; c0 < a.Cout; c0 += 32) {
            const unsigned char* sl = stg + (c0 >> 5) * slice;
            if (!a.upsample) {
                tma_store_4d(tmY, sl, a.y_coff + c0, 0, y0, n0);
            } else {
#pragma unroll
                for (int ab = 0; ab < 4; ++ab) tma_store_5d(tmY, sl, a.y_coff + c0, ab & 1, 0, ab >> 1, n0 * a.H + y0);
            }
        }
        asm volatile("cp.async.bulk.commit_group;" ::: "memory");
        asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
    }
}

__global__ void __launch_bounds__(128, 1)
    conv3x3_tc(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
               const __grid_constant__ CUtensorMap tmY, const ConvArgs a)
{
    extern __shared__ unsigned char smem_raw[];
    if (a.count && (int)((blockIdx.x * kTileM) / (a.H * a.W)) >= *a.count) return;  // no such tile (uniform)
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
        epilogue_store(a, &tmY, tmem, smem, a.bias, 1, n0, y0);
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

// Halo form of the same convolution, for layers whose 128-pixel tile is whole rows of
// one image: a CTA computes R = mt 128 / W whole rows of one image into mt accumulators
// of 128 pixels (mt Cout tensor-memory columns).  A K step is one (channel block, dx)
// pair rather than one (channel block, tap): a single activation box of R + 2 rows x W
// pixels x 32 channels at column offset dx - 1 (rows y0 - 1 and y0 + R and columns -1 and
// W lie outside the image and arrive as zeros) and the three weight boxes of the taps
// (0, dx), (1, dx), (2, dx).  In NHWC the box is R + 2 rows of W pixels of 64 bytes, so
// the operand of tap dy for accumulator j is the same box read from pixel row j 128 +
// dy W: a start (j 128 + dy W) 64 bytes in, a whole number of 512-byte swizzle atoms
// for W a multiple of 8, and the three dy taps share one copy.  Activation bytes copied
// per output pixel: 3 (R + 2) / R boxes instead of 9; weight bytes: 1 / mt of the
// one-tile form.
constexpr int kMaxStages = 4;

__global__ void __launch_bounds__(128, 1)
    conv3x3_halo(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                 const __grid_constant__ CUtensorMap tmY, const ConvArgs a, int nbands)
{
    extern __shared__ unsigned char smem_raw[];
    const int mt = a.mt, S = a.stages;
    const int tile_px = mt * kTileM;
    const int R = tile_px / a.W;
    const int bands_per_tile = a.H / R;
    // bands of tiles at or after *count are skipped (the tile list's length)
    const int live = a.count ? min(nbands, *a.count * bands_per_tile) : nbands;
    if ((int)blockIdx.x >= live) return;  // uniform
    unsigned char* smem = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) &
                                                           ~static_cast<uintptr_t>(1023));
    const int a_bytes = (R + 2) * a.W * kKc * 2;
    const int a_span = (a_bytes + 1023) & ~1023;
    const int b_tap = a.Cout * kKc * 2;
    const int stage_bytes = a_span + ((3 * b_tap + 1023) & ~1023);
    uint64_t* full = reinterpret_cast<uint64_t*>(smem + S * stage_bytes);
    uint64_t* empty = full + kMaxStages;
    uint64_t* done = empty + kMaxStages;
    uint32_t* tslot = reinterpret_cast<uint32_t*>(done + 1);
    volatile int* counts = reinterpret_cast<volatile int*>(tslot + 1);  // [0] issued, [1] consumed, [2] abort
    float* sbias = reinterpret_cast<float*>(smem + S * stage_bytes + 1024);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

    const int cb_n = a.Cin / kKc;
    const int nk = 3 * cb_n;  // K steps of a band: (channel block, dx)
    // K step kk of the CTA (band kk / nk of its walk, step kk % nk) into stage kk % S
    auto issue = [&](int kk, int n0, int y0) {
        const int s = kk % S;
        const int k = kk % nk;
        const int cb = k / 3, dx = k - 3 * cb;
        unsigned char* sa = smem + s * stage_bytes;
        mbar_expect_tx(&full[s], (uint32_t)(a_bytes + 3 * b_tap));
        tma_load_4d(sa, &tmA, &full[s], cb * kKc, dx - 1, y0 - 1, n0);
#pragma unroll
        for (int dy = 0; dy < 3; ++dy)
            tma_load_2d(sa + a_span + dy * b_tap, &tmB, &full[s], (3 * dy + dx) * a.Cin + cb * kKc, 0);
        counts[0] = kk + 1;
    };
    const int first = nk < S ? nk : S;  // copies issued before the CTA-wide barrier

    // The first copies start as soon as the barriers exist (their stages are free), while
    // warp 1 allocates the tensor memory and the bias is staged in shared memory.
    if (threadIdx.x == 0) {
        for (int s = 0; s < S; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        mbar_init(done, 1);
        counts[0] = 0;
        counts[1] = 0;
        counts[2] = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        const int b0 = blockIdx.x, n0 = b0 / bands_per_tile, y0 = (b0 - n0 * bands_per_tile) * R;
        for (int k = 0; k < first; ++k) issue(k, n0, y0);
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tslot)),
                     "r"(a.ncols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    for (int c = threadIdx.x; c < a.Cout; c += blockDim.x) sbias[c] = __ldg(a.bias + c);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tslot;

    // The CTA walks bands blockIdx.x, + gridDim.x, ...: per band its K steps, then the
    // epilogue; the barriers' phases run on across bands (step kk of the walk), and the
    // accumulators are reused once every thread's reads of them are done.
    // Where a band's output fits one stage, the epilogue stages it in the stage of the
    // band's last K step, and the next band's first copy (into the other stage) is issued
    // by the MMA thread once that stage is free, so it lands during the last MMAs and the
    // epilogue.
    const bool early = mt * kTileM * a.Cout * 2 <= stage_bytes && S >= 2;
    int it = 0;
    for (int band = blockIdx.x; band < live; band += gridDim.x, ++it) {
        const int n0 = band / bands_per_tile, y0 = (band - n0 * bands_per_tile) * R;
        const uint64_t deadline = globaltimer() + kWaitNs;
        if (warp == 0 && lane == 0) {  // copies
            for (int k = it == 0 ? first : (early ? 1 : 0); k < nk; ++k) {
                const int kk = it * nk + k, s = kk % S;
                if (!mbar_wait(&empty[s], ((kk / S) & 1) ^ 1, deadline)) {
                    atomicOr(&g_unet_status, kUnetTimeout);
                    counts[2] = 1;
                    break;
                }
                issue(kk, n0, y0);
            }
        } else if (warp == 1 && lane == 0) {  // MMAs
            // Descriptors: a stage's bases plus constants in the 16-byte start-address
            // field (the smem window is below 256 KB, so the field never carries over).
            const uint32_t idesc = idesc_bf16(a.Cout);
            const uint64_t dbase = desc_sw64(smem_u32(smem));
            const uint32_t aW = (uint32_t)a.W * 4u, aT = (uint32_t)kTileM * 4u, bT = (uint32_t)b_tap >> 4;
            const uint32_t d1 = tmem + (uint32_t)a.Cout;
            for (int k = 0; k < nk; ++k) {
                const int kk = it * nk + k, s = kk % S;
                if (!mbar_wait(&full[s], (kk / S) & 1, deadline)) {
                    atomicOr(&g_unet_status, kUnetTimeout);
                    counts[2] = 1;
                    break;
                }
                tc_fence_after();
                const uint64_t da = dbase + (uint64_t)((uint32_t)(s * stage_bytes) >> 4);
                const uint64_t db = da + (uint64_t)((uint32_t)a_span >> 4);
#pragma unroll
                for (int dy = 0; dy < 3; ++dy) {
                    const uint64_t bt = db + dy * bT;
                    const uint64_t a0 = da + dy * aW, a1 = a0 + aT;
                    const uint32_t acc = (k > 0 || dy > 0) ? 1u : 0u;
                    mma_bf16(tmem, a0, bt, idesc, acc);
                    mma_bf16(tmem, a0 + 2, bt + 2, idesc, 1u);
                    mma_bf16(d1, a1, bt, idesc, acc);
                    mma_bf16(d1, a1 + 2, bt + 2, idesc, 1u);
                }
                mma_commit(&empty[s]);
                counts[1] = kk + 1;
            }
            mma_commit(done);  // arrives once every MMA issued above has completed
            // early: the next band's first copy, into the stage the second-to-last K step
            // frees, while this band's last MMAs run
            const int next = band + (int)gridDim.x;
            if (early && next < live && !counts[2]) {
                const int kk = (it + 1) * nk, s = kk % S;
                const int n1 = next / bands_per_tile, y1 = (next - n1 * bands_per_tile) * R;
                if (mbar_wait(&empty[s], ((kk / S) & 1) ^ 1, deadline)) issue(kk, n1, y1);
                else {
                    atomicOr(&g_unet_status, kUnetTimeout);
                    counts[2] = 1;
                }
            }
        }
        __syncwarp();
        const bool ok = mbar_wait(done, it & 1, deadline + kWaitNs);
        if (!ok) {
            atomicOr(&g_unet_status, kUnetTimeout);
            counts[2] = 1;
        }
        __syncthreads();
        const bool go = ok && !counts[2];  // the same for every thread (read after the barrier)
        if (go) {
            tc_fence_after();
            // early: the stage of this band's last K step (its copies were consumed)
            unsigned char* stg = early ? smem + ((it * nk + nk - 1) % S) * stage_bytes : smem;
            epilogue_store(a, &tmY, tmem, stg, sbias, mt, n0, y0);
        }
        // every thread's reads of the accumulators are done before the next band's MMAs
        tc_fence_before();
        __syncthreads();
        tc_fence_after();
        if (!go) break;
    }
    __syncthreads();
    if (threadIdx.x == 0 && counts[2]) {  // copies still in flight after a timeout: wait for them (bounded)
        const uint64_t d2 = globaltimer() + kWaitNs;
        for (int k = counts[1]; k < counts[0]; ++k)
            if (!mbar_wait(&full[k % S], (k / S) & 1, d2)) break;
    }
    __syncthreads();
    if (warp == 1) {  // the allocating warp frees
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

// Halo form: bytes of one copy stage (activation box of R + 2 rows, three weight boxes).
int halo_stage_bytes(int W, int rows, int cout)
{
    return ((((rows + 2) * W * kKc * 2) + 1023) & ~1023) + ((3 * cout * kKc * 2 + 1023) & ~1023);
}

// Halo form: the stages, then 1 KB of barriers and counters, then the bias (256 floats).
size_t halo_smem_bytes(int stage_bytes, int stages)
{
    return 1024 + (size_t)stages * stage_bytes + 1024 + 256 * 4;
}

// Shared memory a halo-form CTA may take: at least two CTAs share an SM (228 KB, 1 KB
// reserved per CTA); with two stages, three fit for Cout <= 64.
constexpr int kHaloSmemBudget = 112 * 1024;

// The halo form's shape for a layer, or mt = 0 where the one-tile form runs: whole-row
// tiles of one image (W in 16..128), two accumulators of 128 pixels (R = 256 / W rows,
// a divisor of H), Cout <= 128 (2 Cout tensor-memory columns), two copy stages within
// the budget.  Two accumulators with two stages (three CTAs per SM for Cout <= 64, two
// for Cout = 128) measured fastest on every layer of the network, against one or four
// accumulators and two to four stages at one to four CTAs per SM: more CTAs per SM
// overlap one CTA's set-up, last MMAs and epilogue with the others' copies.
void halo_shape(int H, int W, int Cout, int* mt, int* stages)
{
    *mt = 0;
    *stages = 0;
    if (W < 16 || W > kTileM || kTileM % W || Cout > 128) return;
    const int rows = 2 * kTileM / W;
    if (rows > H || H % rows) return;
    if (halo_smem_bytes(halo_stage_bytes(W, rows, Cout), 2) > (size_t)kHaloSmemBudget) return;
    if ((Cout / kKc) * 2 * kTileM * 64 > 2 * halo_stage_bytes(W, rows, Cout)) return;  // the epilogue's staging
    *mt = 2;
    *stages = 2;
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
// Shared memory of one SM (228 KB) and the SM count of the current device.
constexpr size_t kSmemPerSm = 228 * 1024;

int sm_count()
{
    static int n = 0;
    if (!n) {
        int dev = 0, v = 0;
        if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) !=
                                                      cudaSuccess || v < 1) {
            cudaGetLastError();
            return 148;
        }
        n = v;
    }
    return n;
}

// Needs T H W a multiple of 128, W in {8, 16, 32, 64, 128} with 128 / W rows per tile or
// whole tiles per 128 pixels, Cout in {32, 64, 128, 256}.  Returns cudaErrorInvalidValue
// for shapes it does not take.
cudaError_t unet_conv3x3(const void* x, int T, int H, int W, int Cin, const void* wk, const float* bias, void* y,
                         int Cout, int y_cstride, int y_coff, int upsample, int relu, cudaStream_t stream,
                         const int* count)
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
    if (reinterpret_cast<uintptr_t>(y) % 16) return cudaErrorInvalidValue;  // a TMA store's base
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

    // The output map: the epilogue's box of 32 channels x the CTA's pixels (rows x W x
    // images), or for the upsampling a 5-D view {channel, b, x, a, n H + y} of the 2H x 2W
    // output with pixel (2y + a, 2x + b), whose box {32, 1, W, 1, rows} takes one replica.
    const cuuint64_t cs = (cuuint64_t)y_cstride;
    auto y_map = [&](CUtensorMap* m, int rows, int imgs) -> bool {
        if (!upsample) {
            const cuuint64_t d[4] = {cs, (cuuint64_t)W, (cuuint64_t)H, (cuuint64_t)T};
            const cuuint64_t st[3] = {cs * 2, (cuuint64_t)W * cs * 2, (cuuint64_t)H * W * cs * 2};
            const cuuint32_t box[4] = {(cuuint32_t)kKc, (cuuint32_t)W, (cuuint32_t)rows, (cuuint32_t)imgs};
            return enc(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, y, d, st, box, one4, CU_TENSOR_MAP_INTERLEAVE_NONE,
                       CU_TENSOR_MAP_SWIZZLE_64B, CU_TENSOR_MAP_L2_PROMOTION_NONE,
                       CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
        }
        const cuuint64_t d[5] = {cs, 2, (cuuint64_t)W, 2, (cuuint64_t)T * H};
        const cuuint64_t st[4] = {cs * 2, 2 * cs * 2, (cuuint64_t)2 * W * cs * 2, (cuuint64_t)4 * W * cs * 2};
        const cuuint32_t box[5] = {(cuuint32_t)kKc, 1, (cuuint32_t)W, 1, (cuuint32_t)(rows * imgs)};
        const cuuint32_t one5[5] = {1, 1, 1, 1, 1};
        return enc(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 5, y, d, st, box, one5, CU_TENSOR_MAP_INTERLEAVE_NONE,
                   CU_TENSOR_MAP_SWIZZLE_64B, CU_TENSOR_MAP_L2_PROMOTION_NONE,
                   CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
    };

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
    a.count = count;
    a.mt = 0;
    a.stages = kStages;
    int mt = 0, stages = 0;
    if (nb == 1) halo_shape(H, W, Cout, &mt, &stages);
    if (mt) {
        const int rows = mt * kTileM / W;
        CUtensorMap th;
        const cuuint32_t hbox[4] = {(cuuint32_t)kKc, (cuuint32_t)W, (cuuint32_t)(rows + 2), 1u};
        if (enc(&th, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, const_cast<void*>(x), adim, astr, hbox, one4,
                CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
            return cudaErrorInvalidValue;
        CUtensorMap ty;
        if (!y_map(&ty, rows, 1)) return cudaErrorInvalidValue;
        a.mt = mt;
        a.stages = stages;
        int nc = 32;
        while (nc < mt * Cout) nc *= 2;
        a.ncols = nc;
        static bool halo_configured = false;
        if (!halo_configured) {
            const cudaError_t e =
                cudaFuncSetAttribute(conv3x3_halo, cudaFuncAttributeMaxDynamicSharedMemorySize, kHaloSmemBudget);
            if (e != cudaSuccess) return e;
            halo_configured = true;
        }
        const size_t hsmem = halo_smem_bytes(halo_stage_bytes(W, rows, Cout), stages);
        // as many CTAs as fit at once (shared memory; registers allow 5), each walking bands
        const int nbands = (int)(pixels / (mt * kTileM));
        const int per_sm = std::min(5, (int)(kSmemPerSm / (hsmem + 1024)));
        const int grid = std::min(nbands, std::max(per_sm, 1) * sm_count());
        conv3x3_halo<<<(unsigned)grid, 128, hsmem, stream>>>(th, tb, ty, a, nbands);
        return cudaGetLastError();
    }
    const size_t smem = conv_smem_bytes(Cout);
    static bool configured = false;
    if (!configured) {
        const cudaError_t e =
            cudaFuncSetAttribute(conv3x3_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)conv_smem_bytes(256));
        if (e != cudaSuccess) return e;
        configured = true;
    }
    CUtensorMap ty;
    if (!y_map(&ty, hb, nb)) return cudaErrorInvalidValue;
    conv3x3_tc<<<(unsigned)(pixels / kTileM), 128, smem, stream>>>(ta, tb, ty, a);
    return cudaGetLastError();
}

namespace {

constexpr int kTile = 64;  // inference tile: 64 x 64 pixels
constexpr int kInCh = 6;   // network input channels (padded to 32 in memory)
constexpr int kLevels = 4;
constexpr int kWidths[kLevels] = {32, 64, 128, 256};

// ---- small CUDA-core kernels around the convolutions

// The frames of one inpainting launch.  Their cell grids are concatenated: cell c of frame
// f (c = ty * ntx + tx) is entry off[f] + c, so their hole cells form one list and one pass
// of the network takes them all.
constexpr int kMaxInpaintFrames = 32;

struct FrameTable {
    int n;
    int off[kMaxInpaintFrames + 1];  // off[n]: cells of all frames
    int w[kMaxInpaintFrames], h[kMaxInpaintFrames], ntx[kMaxInpaintFrames];
    float near_[kMaxInpaintFrames];
    uint32_t* rgba[kMaxInpaintFrames];
    const uint8_t* mask[kMaxInpaintFrames];
    const float* zt[kMaxInpaintFrames];
    const float* zsrc[kMaxInpaintFrames];
};

// Frame of concatenated cell g.
__device__ __forceinline__ int table_frame(const FrameTable& ft, int g)
{
    int lo = 0, hi = ft.n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (ft.off[mid] <= g) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// Per 64 x 64 cell of each frame (blockIdx.x: cell, blockIdx.y: frame): 1 if it holds a
// hole pixel (mask == 1), at the cell's entry of the concatenated grids.
__global__ void tile_flags_kernel(const __grid_constant__ FrameTable ft, int* __restrict__ flags)
{
    const int f = blockIdx.y, cell = blockIdx.x;
    const int w = ft.w[f], h = ft.h[f], ntx = ft.ntx[f];
    if (cell >= ntx * ((h + kTile - 1) / kTile)) return;  // uniform
    const int tx = cell % ntx, ty = cell / ntx;
    const uint8_t* mask = ft.mask[f];
    int any = 0;
    for (int i = threadIdx.x; i < kTile * kTile; i += blockDim.x) {
        const int x = tx * kTile + (i & (kTile - 1)), y = ty * kTile + (i >> 6);
        if (x < w && y < h && mask[(size_t)y * w + x]) any = 1;
    }
    any = __syncthreads_or(any);
    if (threadIdx.x == 0) flags[ft.off[f] + cell] = any;
}

// Ordered list of the flagged tiles (index ty * ntx + tx) and its length, one CTA.
__global__ void tile_list_kernel(const int* __restrict__ flags, int ntiles, int* __restrict__ list,
                                 int* __restrict__ count)
{
    __shared__ int warp_sums[32];
    __shared__ int base;
    if (threadIdx.x == 0) base = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int c0 = 0; c0 < ntiles; c0 += blockDim.x) {
        const int i = c0 + threadIdx.x;
        const int f = i < ntiles ? flags[i] : 0;
        int incl = f;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int v = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += v;
        }
        if (lane == 31) warp_sums[warp] = incl;
        __syncthreads();
        if (warp == 0) {
            const int nw = blockDim.x >> 5;
            int ws = lane < nw ? warp_sums[lane] : 0;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int v = __shfl_up_sync(0xffffffffu, ws, o);
                if (lane >= o) ws += v;
            }
            if (lane < nw) warp_sums[lane] = ws;  // inclusive prefix of warp totals
        }
        __syncthreads();
        const int before = base + (warp ? warp_sums[warp - 1] : 0) + incl - f;
        if (f) list[before] = i;
        __syncthreads();
        if (threadIdx.x == blockDim.x - 1) base = before + f;
        __syncthreads();
    }
    if (threadIdx.x == 0) *count = base;
}

__device__ __forceinline__ uint16_t bf16_bits(float v)
{
    const __nv_bfloat16 b = __float2bfloat16_rn(v);
    return *reinterpret_cast<const uint16_t*>(&b);
}

// Origin of the 64 x 64 window of grid cell (tx, ty): the cell itself, except that the
// last column and row are shifted inward so the window ends at the frame's edge (a frame
// narrower or lower than 64 keeps origin 0 and is padded).  A tile writes its cell only.
__device__ __forceinline__ int window_origin(int t, int size) { return max(0, min(kTile * t, size - kTile)); }

// The network input of listed tile ti, pixel (py, px) of its window: the six channels of
// the definition (the plain path's right eye / 255: warped colors and the Patcher's fill
// at holes; the hole mask; near / warped depth, 0 at holes; near / source depth), rounded
// to bfloat16, then 26 zero channels.
// Pixels outside the frame (frames smaller than a tile) are all zero.
__global__ void tile_input_kernel(const __grid_constant__ FrameTable ft, const int* __restrict__ list,
                                  const int* __restrict__ count, uint16_t* __restrict__ x)
{
    const int ti = blockIdx.y;
    if (ti >= *count) return;
    const int p = blockIdx.x * blockDim.x + threadIdx.x;  // pixel of the tile
    if (p >= kTile * kTile) return;
    const int g = list[ti];
    const int f = table_frame(ft, g);
    const int tile = g - ft.off[f];
    const int w = ft.w[f], h = ft.h[f], ntx = ft.ntx[f];
    const float near_ = ft.near_[f];
    const int gx = window_origin(tile % ntx, w) + (p & (kTile - 1)), gy = window_origin(tile / ntx, h) + (p >> 6);
    float c[kInCh] = {0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f};
    if (gx < w && gy < h) {
        const size_t o = (size_t)gy * w + gx;
        const bool hole = ft.mask[f][o] != 0;
        const uint32_t v = ft.rgba[f][o];
        c[0] = __fdiv_rn((float)(v & 255u), 255.0f);
        c[1] = __fdiv_rn((float)((v >> 8) & 255u), 255.0f);
        c[2] = __fdiv_rn((float)((v >> 16) & 255u), 255.0f);
        if (!hole) c[4] = __fdiv_rn(near_, fmaxf(ft.zt[f][o], near_));
        c[3] = hole ? 1.0f : 0.0f;
        c[5] = __fdiv_rn(near_, fmaxf(ft.zsrc[f][o], near_));
    }
    uint4 q[4] = {};
    uint32_t* qw = reinterpret_cast<uint32_t*>(q);
    qw[0] = (uint32_t)bf16_bits(c[0]) | ((uint32_t)bf16_bits(c[1]) << 16);
    qw[1] = (uint32_t)bf16_bits(c[2]) | ((uint32_t)bf16_bits(c[3]) << 16);
    qw[2] = (uint32_t)bf16_bits(c[4]) | ((uint32_t)bf16_bits(c[5]) << 16);
    uint4* dst = reinterpret_cast<uint4*>(x + ((size_t)ti * kTile * kTile + p) * 32);
#pragma unroll
    for (int i = 0; i < 4; ++i) dst[i] = q[i];
}

// 2x2 max pooling of channels [0, C) of x (T x H x W, cstride channels) into y (T x H/2 x
// W/2 x C), eight channels per thread.  bfloat16 values compare exactly as floats.
__global__ void maxpool_kernel(const uint16_t* __restrict__ x, int T, int H, int W, int cstride, int C,
                               uint16_t* __restrict__ y, const int* __restrict__ count)
{
    const int Ho = H / 2, Wo = W / 2, cv = C / 8;
    const long long total = (long long)T * Ho * Wo * cv;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const int v = (int)(i % cv);
        long long r = i / cv;
        const int xo = (int)(r % Wo);
        r /= Wo;
        const int yo = (int)(r % Ho);
        const int t = (int)(r / Ho);
        if (count && t >= *count) continue;
        float m[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) m[k] = -INFINITY;
#pragma unroll
        for (int ab = 0; ab < 4; ++ab) {
            const size_t px = ((size_t)t * H + 2 * yo + (ab >> 1)) * W + 2 * xo + (ab & 1);
            const uint4 q = *reinterpret_cast<const uint4*>(x + px * cstride + v * 8);
            const uint32_t qw[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
            for (int k = 0; k < 8; ++k)
                m[k] = fmaxf(m[k], __uint_as_float((k & 1 ? qw[k >> 1] & 0xffff0000u : qw[k >> 1] << 16)));
        }
        uint4 o;
        uint32_t* ow = reinterpret_cast<uint32_t*>(&o);
#pragma unroll
        for (int k = 0; k < 4; ++k)
            ow[k] = (__float_as_uint(m[2 * k]) >> 16) | (__float_as_uint(m[2 * k + 1]) & 0xffff0000u);
        *reinterpret_cast<uint4*>(y + (((size_t)t * Ho + yo) * Wo + xo) * C + v * 8) = o;
    }
}

// The output layer at pixel p of tile ti: a 1x1 convolution of the 32 channels (FP32 sums
// in channel order, then the bias) and the logistic sigmoid 1 / (1 + exp(-z)).
__device__ __forceinline__ void net_colors(const uint16_t* __restrict__ a, const float* __restrict__ wo,
                                           const float* __restrict__ bo, int ti, int p, float (&col)[3])
{
    const uint4* src = reinterpret_cast<const uint4*>(a + ((size_t)ti * kTile * kTile + p) * 32);
    float v[32];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const uint4 q = src[i];
        const uint32_t qw[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            v[8 * i + 2 * k] = __uint_as_float(qw[k] << 16);
            v[8 * i + 2 * k + 1] = __uint_as_float(qw[k] & 0xffff0000u);
        }
    }
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        float acc = 0.0f;
#pragma unroll
        for (int ci = 0; ci < 32; ++ci) acc = __fadd_rn(acc, __fmul_rn(wo[c * 32 + ci], v[ci]));
        const float z = __fadd_rn(acc, bo[c]);
        col[c] = __fdiv_rn(1.0f, __fadd_rn(1.0f, expf(-z)));
    }
}

// The three colors of every pixel of the first T tiles to rgb (T x 64 x 64 x 3 floats).
__global__ void output_kernel(const uint16_t* __restrict__ a, const float* __restrict__ wo,
                              const float* __restrict__ bo, int T, float* __restrict__ rgb)
{
    const int ti = blockIdx.y;
    if (ti >= T) return;
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= kTile * kTile) return;
    float col[3];
    net_colors(a, wo, bo, ti, p, col);
    float* o = rgb + ((size_t)ti * kTile * kTile + p) * 3;
    o[0] = col[0];
    o[1] = col[1];
    o[2] = col[2];
}

// Compose into the frames: each hole pixel of a listed tile's cell takes rint(clamp(c, 0,
// 1) * 255) per color and alpha 255 (the pixels of the window outside the cell belong to
// the neighbouring tile).
__global__ void compose_kernel(const uint16_t* __restrict__ a, const float* __restrict__ wo,
                               const float* __restrict__ bo, const int* __restrict__ count,
                               const int* __restrict__ list, const __grid_constant__ FrameTable ft)
{
    const int ti = blockIdx.y;
    if (ti >= *count) return;
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= kTile * kTile) return;
    const int g = list[ti];
    const int f = table_frame(ft, g);
    const int tile = g - ft.off[f];
    const int w = ft.w[f], h = ft.h[f], ntx = ft.ntx[f];
    const int tx = tile % ntx, ty = tile / ntx;
    const int gx = window_origin(tx, w) + (p & (kTile - 1)), gy = window_origin(ty, h) + (p >> 6);
    if (gx < kTile * tx || gy < kTile * ty || gx >= w || gy >= h || !ft.mask[f][(size_t)gy * w + gx]) return;
    float col[3];
    net_colors(a, wo, bo, ti, p, col);
    uint32_t out = 0xff000000u;
#pragma unroll
    for (int c = 0; c < 3; ++c)
        out |= (uint32_t)rintf(__fmul_rn(fminf(fmaxf(col[c], 0.0f), 1.0f), 255.0f)) << (8 * c);
    ft.rgba[f][(size_t)gy * w + gx] = out;
}

void host_bf16_impl(const float* src, size_t n, uint16_t* dst)
{
    for (size_t i = 0; i < n; ++i) {
        uint32_t u;
        std::memcpy(&u, &src[i], 4);
        if ((u & 0x7fffffffu) > 0x7f800000u) {  // NaN stays NaN
            dst[i] = (uint16_t)((u >> 16) | 0x40u);
            continue;
        }
        u += 0x7fffu + ((u >> 16) & 1u);
        dst[i] = (uint16_t)(u >> 16);
    }
}

}  // namespace

void host_bf16(const float* src, size_t n, uint16_t* dst) { host_bf16_impl(src, n, dst); }

cudaError_t unet_output_rgb(const UnetNet* n, int T, float* rgb, cudaStream_t s)
{
    output_kernel<<<dim3(16, (unsigned)T), 256, 0, s>>>(n->d0b, n->wout, n->wout + 96, T, rgb);
    return cudaGetLastError();
}

size_t unet_param_count()
{
    size_t n = 0;
    int cin = kInCh;
    for (int l = 0; l < kLevels; ++l) {
        n += (size_t)kWidths[l] * cin * 9 + kWidths[l] + (size_t)kWidths[l] * kWidths[l] * 9 + kWidths[l];
        cin = kWidths[l];
    }
    for (int l = kLevels - 2; l >= 0; --l) {
        const int c = kWidths[l];
        n += (size_t)c * (c + kWidths[l + 1]) * 9 + c + (size_t)c * c * 9 + c;
    }
    return n + 3 * 32 + 3;
}

void unet_layer_dims(int i, int* cin, int* cout)
{
    // i = 0..7 encoder (level i / 2), 8..13 decoder (levels 2, 1, 0)
    if (i < 8) {
        const int l = i / 2;
        *cout = kWidths[l];
        *cin = (i % 2) ? kWidths[l] : (l ? kWidths[l - 1] : kInCh);
    } else {
        const int l = 2 - (i - 8) / 2;
        *cout = kWidths[l];
        *cin = ((i - 8) % 2) ? kWidths[l] : kWidths[l] + kWidths[l + 1];
    }
}

void unet_free(UnetNet* n)
{
    if (!n) return;
    for (auto& L : n->conv) {
        cudaFree(L.wk);
        cudaFree(L.bias);
    }
    cudaFree(n->wout);
    uint16_t* bufs[] = {n->in0, n->e0a, n->cat0, n->p0, n->e1a, n->cat1, n->p1, n->e2a,
                        n->cat2, n->p2, n->e3a, n->d2a, n->d1a, n->d0a, n->d0b};
    for (uint16_t* b : bufs) cudaFree(b);
    cudaFree(n->flags);
    cudaFree(n->list);
    cudaFree(n->count);
    delete n;
}

UnetNet* unet_create(const float* params, size_t n_params, int max_tiles, int max_grid_tiles)
{
    if (!params || n_params != unet_param_count() || max_tiles < 1 || max_grid_tiles < 1) return nullptr;
    UnetNet* n = new UnetNet();
    std::memset(n, 0, sizeof *n);
    n->max_tiles = (max_tiles + 1) & ~1;  // even: the 8 x 8 level takes two tiles per 128-pixel MMA tile
    n->max_grid_tiles = max_grid_tiles;
    bool ok = true;
    const float* p = params;
    std::vector<uint16_t> hk;
    for (int i = 0; i < 14 && ok; ++i) {
        int cin, cout;
        unet_layer_dims(i, &cin, &cout);
        UnetLayer& L = n->conv[i];
        L.cin = cin;
        L.cout = cout;
        L.cin_pad = (cin + 31) / 32 * 32;
        // (cout, cin, 3, 3) -> (cout, 3, 3, cin_pad), bfloat16
        std::vector<float> km((size_t)cout * 9 * L.cin_pad, 0.0f);
        for (int co = 0; co < cout; ++co)
            for (int ci = 0; ci < cin; ++ci)
                for (int t = 0; t < 9; ++t) km[((size_t)co * 9 + t) * L.cin_pad + ci] = p[((size_t)co * cin + ci) * 9 + t];
        p += (size_t)cout * cin * 9;
        hk.resize(km.size());
        host_bf16(km.data(), km.size(), hk.data());
        ok = cudaMalloc(&L.wk, hk.size() * 2) == cudaSuccess && cudaMalloc(&L.bias, cout * 4) == cudaSuccess &&
             cudaMemcpy(L.wk, hk.data(), hk.size() * 2, cudaMemcpyHostToDevice) == cudaSuccess &&
             cudaMemcpy(L.bias, p, cout * 4, cudaMemcpyHostToDevice) == cudaSuccess;
        p += cout;
    }
    if (ok) {  // output layer: bfloat16-rounded weights kept as floats, FP32 biases
        std::vector<uint16_t> b16(96);
        host_bf16(p, 96, b16.data());
        float wo[99];
        for (int i = 0; i < 96; ++i) {
            const uint32_t u = (uint32_t)b16[i] << 16;
            std::memcpy(&wo[i], &u, 4);
        }
        for (int i = 0; i < 3; ++i) wo[96 + i] = p[96 + i];
        ok = cudaMalloc(&n->wout, sizeof wo) == cudaSuccess &&
             cudaMemcpy(n->wout, wo, sizeof wo, cudaMemcpyHostToDevice) == cudaSuccess;
    }
    const size_t T = n->max_tiles, P0 = T * 64 * 64, P1 = T * 32 * 32, P2 = T * 16 * 16, P3 = T * 8 * 8;
    struct {
        uint16_t** b;
        size_t elems;
    } al[] = {{&n->in0, P0 * 32}, {&n->e0a, P0 * 32}, {&n->cat0, P0 * 96}, {&n->p0, P1 * 32}, {&n->e1a, P1 * 64},
              {&n->cat1, P1 * 192}, {&n->p1, P2 * 64}, {&n->e2a, P2 * 128}, {&n->cat2, P2 * 384},
              {&n->p2, P3 * 128}, {&n->e3a, P3 * 256}, {&n->d2a, P2 * 128}, {&n->d1a, P1 * 64},
              {&n->d0a, P0 * 32}, {&n->d0b, P0 * 32}};
    for (auto& x : al)
        if (ok) ok = cudaMalloc(x.b, x.elems * 2) == cudaSuccess;
    if (ok) {
        // the in0 buffer of tiles never written stays zero (T rounded up to even)
        ok = cudaMemset(n->in0, 0, P0 * 32 * 2) == cudaSuccess &&
             cudaMalloc(&n->flags, (size_t)max_grid_tiles * 4) == cudaSuccess &&
             cudaMalloc(&n->list, (size_t)max_grid_tiles * 4) == cudaSuccess &&
             cudaMalloc(&n->count, 4) == cudaSuccess;
    }
    if (!ok) {
        cudaGetLastError();
        unet_free(n);
        return nullptr;
    }
    return n;
}

// The 14 convolutions and the pools over the first T tiles of in0 (tiles at or after
// *count skipped when count is given); the last layer's activations end in d0b.
cudaError_t unet_run(UnetNet* n, int T, const int* count, cudaStream_t s)
{
    const int Te = (T + 1) & ~1;
    cudaError_t e = cudaSuccess;
    auto conv = [&](int i, const uint16_t* x, int H, void* y, int cstride, int coff, int up) {
        if (e != cudaSuccess) return;
        const UnetLayer& L = n->conv[i];
        e = unet_conv3x3(x, Te, H, H, L.cin_pad, L.wk, L.bias, y, L.cout, cstride, coff, up, 1, s, count);
    };
    auto pool = [&](const uint16_t* x, int H, int cstride, int C, uint16_t* y) {
        if (e != cudaSuccess) return;
        const long long total = (long long)Te * (H / 2) * (H / 2) * (C / 8);
        const int blocks = (int)std::min<long long>((total + 255) / 256, 4096);
        maxpool_kernel<<<blocks, 256, 0, s>>>(x, Te, H, H, cstride, C, y, count);
        e = cudaGetLastError();
    };
    conv(0, n->in0, 64, n->e0a, 32, 0, 0);     // enc0a
    conv(1, n->e0a, 64, n->cat0, 96, 0, 0);    // enc0b -> skip of level 0
    pool(n->cat0, 64, 96, 32, n->p0);
    conv(2, n->p0, 32, n->e1a, 64, 0, 0);      // enc1a
    conv(3, n->e1a, 32, n->cat1, 192, 0, 0);   // enc1b -> skip of level 1
    pool(n->cat1, 32, 192, 64, n->p1);
    conv(4, n->p1, 16, n->e2a, 128, 0, 0);     // enc2a
    conv(5, n->e2a, 16, n->cat2, 384, 0, 0);   // enc2b -> skip of level 2
    pool(n->cat2, 16, 384, 128, n->p2);
    conv(6, n->p2, 8, n->e3a, 256, 0, 0);      // enc3a
    conv(7, n->e3a, 8, n->cat2, 384, 128, 1);  // enc3b, upsampled after the level-2 skip
    conv(8, n->cat2, 16, n->d2a, 128, 0, 0);   // dec2a
    conv(9, n->d2a, 16, n->cat1, 192, 64, 1);  // dec2b, upsampled after the level-1 skip
    conv(10, n->cat1, 32, n->d1a, 64, 0, 0);   // dec1a
    conv(11, n->d1a, 32, n->cat0, 96, 32, 1);  // dec1b, upsampled after the level-0 skip
    conv(12, n->cat0, 64, n->d0a, 32, 0, 0);   // dec0a
    conv(13, n->d0a, 64, n->d0b, 32, 0, 0);    // dec0b
    return e;
}

}  // namespace yoro

struct yoro_unet_ctx {
    yoro::UnetNet* net;
    int device;
    int max_w, max_h;
};

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

long long yoro_unet_param_count(void) { return (long long)yoro::unet_param_count(); }

yoro_unet yoro_unet_create(const float* params, long long n_params, int max_tiles, int max_w, int max_h)
{
    if (!params || n_params <= 0 || max_tiles < 0 || max_w < 0 || max_h < 0 || max_w > 65536 || max_h > 65536)
        return nullptr;
    const int grid_tiles = ((max_w + 63) / 64) * ((max_h + 63) / 64);
    const int tiles = std::max(std::max(max_tiles, grid_tiles), 2);
    yoro_unet_ctx* c = new (std::nothrow) yoro_unet_ctx();
    if (!c) return nullptr;
    if (cudaGetDevice(&c->device) != cudaSuccess) {
        cudaGetLastError();
        delete c;
        return nullptr;
    }
    c->max_w = max_w;
    c->max_h = max_h;
    c->net = yoro::unet_create(params, (size_t)n_params, tiles, tiles);  // flags and list hold `tiles` cells
    if (!c->net) {
        delete c;
        return nullptr;
    }
    return c;
}

void yoro_unet_destroy(yoro_unet u)
{
    if (!u) return;
    yoro::unet_free(u->net);
    delete u;
}

yoro_status yoro_unet_forward(yoro_unet u, const void* x, int T, float* rgb, void* cuda_stream)
{
    if (!u || !x || !rgb || T < 0 || T > u->net->max_tiles) return YORO_EINVAL;
    if (T == 0) return YORO_OK;
    if (((uintptr_t)x & 15u) || ((uintptr_t)rgb & 3u)) return YORO_EALIGN;
    const cudaStream_t s = (cudaStream_t)cuda_stream;
    if (cudaMemcpyAsync(u->net->in0, x, (size_t)T * 64 * 64 * 32 * 2, cudaMemcpyDeviceToDevice, s) != cudaSuccess)
        return YORO_ECUDA;
    if (yoro::unet_run(u->net, T, nullptr, s) != cudaSuccess) return YORO_ECUDA;
    yoro::output_kernel<<<dim3(16, (unsigned)T), 256, 0, s>>>(u->net->d0b, u->net->wout, u->net->wout + 96, T, rgb);
    return cudaGetLastError() == cudaSuccess ? YORO_OK : YORO_ECUDA;
}

}  // extern "C"

namespace {

// Checks of one frame of the inpainting entry points; YORO_OK, or the status to return.
yoro_status check_frame(const yoro_unet_ctx* u, int w, int h, float near_, const void* rgba,
                        const unsigned char* mask, const float* zt, const float* src_depth)
{
    if (w < 0 || h < 0 || !(near_ > 0.0f) || !std::isfinite(near_)) return YORO_EINVAL;
    if ((size_t)w * h == 0) return YORO_OK;
    if (w > u->max_w || h > u->max_h) return YORO_ETOOBIG;
    if (!rgba || !mask || !zt || !src_depth) return YORO_EINVAL;
    if (((uintptr_t)rgba | (uintptr_t)zt | (uintptr_t)src_depth) & 3u) return YORO_EALIGN;
    return YORO_OK;
}

// Appends frame i to the table (its cells after those already there).
void table_add(yoro::FrameTable& ft, const yoro_unet_frame& fr)
{
    const int k = ft.n;
    ft.w[k] = fr.w;
    ft.h[k] = fr.h;
    ft.ntx[k] = (fr.w + 63) / 64;
    ft.near_[k] = fr.near_;
    ft.rgba[k] = static_cast<uint32_t*>(fr.rgba);
    ft.mask[k] = fr.mask;
    ft.zt[k] = fr.zt;
    ft.zsrc[k] = fr.src_depth;
    ft.off[k + 1] = ft.off[k] + ft.ntx[k] * ((fr.h + 63) / 64);
    ft.n = k + 1;
}

// One pass of the network over the hole cells of the table's frames: the cells' flags, the
// list of the flagged ones and its length on the device (launches cover every cell; those
// past the list's length return at once), the inputs, the 14 layers, the composition.
yoro_status inpaint_table(yoro_unet_ctx* u, const yoro::FrameTable& ft, cudaStream_t s)
{
    yoro::UnetNet* n = u->net;
    const int total = ft.off[ft.n];
    int maxcells = 0;
    for (int f = 0; f < ft.n; ++f) maxcells = std::max(maxcells, ft.off[f + 1] - ft.off[f]);
    if (total == 0) return YORO_OK;
    yoro::tile_flags_kernel<<<dim3((unsigned)maxcells, (unsigned)ft.n), 256, 0, s>>>(ft, n->flags);
    yoro::tile_list_kernel<<<1, 1024, 0, s>>>(n->flags, total, n->list, n->count);
    yoro::tile_input_kernel<<<dim3(16, (unsigned)total), 256, 0, s>>>(ft, n->list, n->count, n->in0);
    if (cudaGetLastError() != cudaSuccess) return YORO_ECUDA;
    if (yoro::unet_run(n, total, n->count, s) != cudaSuccess) return YORO_ECUDA;
    yoro::compose_kernel<<<dim3(16, (unsigned)total), 256, 0, s>>>(n->d0b, n->wout, n->wout + 96, n->count, n->list,
                                                                 ft);
    return cudaGetLastError() == cudaSuccess ? YORO_OK : YORO_ECUDA;
}

}  // namespace

extern "C" {

yoro_status yoro_unet_inpaint(yoro_unet u, int w, int h, float near_, void* rgba, const unsigned char* mask,
                              const float* zt, const float* src_depth, void* cuda_stream)
{
    if (!u) return YORO_EINVAL;
    const yoro_status st = check_frame(u, w, h, near_, rgba, mask, zt, src_depth);
    if (st != YORO_OK || (size_t)w * h == 0) return st;
    yoro::FrameTable ft;
    ft.n = 0;
    ft.off[0] = 0;
    table_add(ft, yoro_unet_frame{w, h, near_, rgba, mask, zt, src_depth});
    return inpaint_table(u, ft, (cudaStream_t)cuda_stream);
}

yoro_status yoro_unet_inpaint_batch(yoro_unet u, int n, const yoro_unet_frame* frames, void* cuda_stream)
{
    if (!u || n < 0 || (n > 0 && !frames)) return YORO_EINVAL;
    for (int i = 0; i < n; ++i) {
        const yoro_unet_frame& fr = frames[i];
        const yoro_status st = check_frame(u, fr.w, fr.h, fr.near_, fr.rgba, fr.mask, fr.zt, fr.src_depth);
        if (st != YORO_OK) return st;
    }
    // groups of frames whose cells fit the network's buffers, up to kMaxInpaintFrames each
    const int capacity = std::min(u->net->max_tiles, u->net->max_grid_tiles);
    yoro::FrameTable ft;
    ft.n = 0;
    ft.off[0] = 0;
    for (int i = 0; i < n; ++i) {
        const yoro_unet_frame& fr = frames[i];
        if ((size_t)fr.w * fr.h == 0) continue;
        const int cells = ((fr.w + 63) / 64) * ((fr.h + 63) / 64);
        if (ft.n == yoro::kMaxInpaintFrames || (ft.n > 0 && ft.off[ft.n] + cells > capacity)) {
            const yoro_status st = inpaint_table(u, ft, (cudaStream_t)cuda_stream);
            if (st != YORO_OK) return st;
            ft.n = 0;
        }
        table_add(ft, fr);
    }
    return ft.n ? inpaint_table(u, ft, (cudaStream_t)cuda_stream) : YORO_OK;
}

yoro_status yoro_unet_prepare(yoro_unet u, int w, int h, float near_, const void* rgba, const unsigned char* mask,
                              const float* zt, const float* src_depth, void* x_out, int max_out, int* list_host,
                              int* count_host, void* cuda_stream)
{
    if (!u || !list_host || !count_host) return YORO_EINVAL;
    *count_host = 0;
    yoro_status st = check_frame(u, w, h, near_, rgba, mask, zt, src_depth);
    if (st != YORO_OK || (size_t)w * h == 0) return st;
    const int ntx = (w + 63) / 64, nty = (h + 63) / 64;
    if (!x_out || max_out < ntx * nty) return YORO_EINVAL;
    if ((uintptr_t)x_out & 15u) return YORO_EALIGN;
    yoro::UnetNet* n = u->net;
    const cudaStream_t s = (cudaStream_t)cuda_stream;
    yoro::FrameTable ft;
    ft.n = 0;
    ft.off[0] = 0;
    table_add(ft, yoro_unet_frame{w, h, near_, const_cast<void*>(rgba), mask, zt, src_depth});
    yoro::tile_flags_kernel<<<dim3((unsigned)(ntx * nty), 1), 256, 0, s>>>(ft, n->flags);
    yoro::tile_list_kernel<<<1, 1024, 0, s>>>(n->flags, ntx * nty, n->list, n->count);
    yoro::tile_input_kernel<<<dim3(16, (unsigned)(ntx * nty)), 256, 0, s>>>(ft, n->list, n->count,
                                                                          static_cast<uint16_t*>(x_out));
    if (cudaGetLastError() != cudaSuccess) return YORO_ECUDA;
    if (cudaMemcpyAsync(count_host, n->count, 4, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaMemcpyAsync(list_host, n->list, (size_t)ntx * nty * 4, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess) {
        cudaGetLastError();
        return YORO_ECUDA;
    }
    return YORO_OK;
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
