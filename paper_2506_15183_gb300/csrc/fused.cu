// Fused second-eye synthesis kernel for GB300 (sm_103a).
//
// One CTA owns a band of output rows.  It streams the band's source rows, plus one
// halo row above and below, through shared memory and runs the whole path per row:
//
//   P1  disparity + forward warp (Alg. 1 closed form, Alg. 2 nearest kept): the
//       row's depth arrives by a 1-D bulk copy (cp.async.bulk, mbarrier-tracked,
//       issued S rows ahead); every source pixel does a 64-bit atomicMin of
//       (depth bits << 32 | source column) into the row's shared-memory z-buffer.
//       Rows are independent (O1: motion is horizontal), so the scatter never
//       leaves the row.
//   P2  resolve + gather: each z-buffer entry becomes (depth, RGBA8 of its source)
//       in place, the source color coming from the staged color row; a warp ballot
//       packs the row's reached/hole flags into a bitmask.
//   P3  hole fill of the row above (Alg. 3, Eq. 6), which needs the warped rows
//       v-1, v, v+1 that the ring of four z-buffer slots keeps: hole edges L/R come
//       from the bitmask (count-leading/trailing-zeros over 32-pixel words), each
//       warp compacts the holes of its 128-pixel blocks so that all 32 lanes fill,
//       candidates are enumerated from the bitmask highest column first, and the
//       finished row leaves by 16-byte stores.
//
// Two barriers per row: P1 | P2 (+ clear the next slot) | P3 (+ issue the next bulk
// copy).  HBM sees 8 B read and 5 B written per pixel plus the two halo rows, which
// neighbouring CTAs read at about the same time (L2).  Every wait on an mbarrier is
// bounded; on expiry the CTA records an error in the status word, waits (bounded)
// for its own copies in flight and leaves.
#include <cuda_runtime.h>

#include <cstdint>

#include "yoro_device.cuh"
#include "yoro_internal.h"

namespace yoro {

namespace {

constexpr int kStages = 2;          // bulk-copy prefetch depth (rows)
constexpr int kWaitLimit = 1 << 20; // polls of an mbarrier before giving up

__device__ __forceinline__ uint32_t smem_addr(const void* p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait: true when the phase with this parity has completed.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity)
{
    for (int i = 0; i < kWaitLimit; ++i)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}

__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_addr(dst)),
        "l"(src), "r"(bytes), "r"(smem_addr(bar))
        : "memory");
}

// Shared-memory carve-up for frames up to `wcap` pixels wide (wcap % 128 == 0).
struct Smem {
    unsigned long long* keys;  // [4][wcap]  z-buffer keys, then (depth, rgba) pairs
    uint32_t* bits;            // [4][wcap/32] reached flags
    uint32_t* outrow;          // [wcap]     finished row before the global store
    float* sdepth;             // [kStages][wcap]
    uint32_t* scolor;          // [kStages][wcap]
    uint64_t* bar;             // [kStages]
    int* flag;                 // [4]        flag[0]: abort
    __device__ Smem(unsigned char* base, int wcap)
    {
        size_t o = 0;
        keys = (unsigned long long*)(base + o);
        o += (size_t)4 * wcap * 8;
        bits = (uint32_t*)(base + o);
        o += (size_t)4 * (wcap / 32) * 4;
        outrow = (uint32_t*)(base + o);
        o += (size_t)wcap * 4;
        sdepth = (float*)(base + o);
        o += (size_t)kStages * wcap * 4;
        scolor = (uint32_t*)(base + o);
        o += (size_t)kStages * wcap * 4;
        bar = (uint64_t*)(base + o);
        o += (size_t)kStages * 8;
        flag = (int*)(base + o);
    }
};

// Hole fill of pixel (v, x); rows v-1, v, v+1 are given as (pairs, bits) or null
// when outside the image.  Pairs are (depth bits, rgba) per reached column.
__device__ __forceinline__ uint32_t fill_pixel(int x, int w, int nwords, const uint2* const pr[3],
                                               const uint32_t* const br[3])
{
    const uint32_t* bv = br[1];
    const uint2* pv = pr[1];
    // L: highest reached column < x.
    int L = -1;
    {
        int wi = x >> 5;
        uint32_t m = bv[wi] & ((1u << (x & 31)) - 1u);
        for (;;) {
            if (m) {
                L = (wi << 5) + 31 - __clz(m);
                break;
            }
            if (--wi < 0) break;
            m = bv[wi];
        }
    }
    // R: lowest reached column > x (bits past the row end are zero).
    int R = w;
    {
        int wi = x >> 5;
        uint32_t m = ((x & 31) == 31) ? 0u : (bv[wi] & (~0u << ((x & 31) + 1)));
        for (;;) {
            if (m) {
                R = (wi << 5) + __ffs(m) - 1;
                break;
            }
            if (++wi >= nwords) break;
            m = bv[wi];
        }
    }
    if (R < w) {
        const int wd = R - L;
        const float d_occ = (L >= 0) ? __uint_as_float(pv[L].x) : 0.0f;
        FillAcc f;
        f.init(__fdiv_rn((float)(R - x), (float)wd));
        const int jhi = min(R + wd, w - 1);
        const int whi = jhi >> 5, wlo = R >> 5;
        const uint32_t mhi = ((jhi & 31) == 31) ? ~0u : ((2u << (jhi & 31)) - 1u);
        const uint32_t mlo = ~0u << (R & 31);
        bool live = true;
#pragma unroll 1
        for (int k = 0; k < 3 && live; ++k) {
            const uint32_t* b = br[k];
            if (b == nullptr) continue;
            const uint2* p = pr[k];
#pragma unroll 1
            for (int wi = whi; wi >= wlo && live; --wi) {
                uint32_t m = b[wi];
                if (wi == whi) m &= mhi;
                if (wi == wlo) m &= mlo;
                while (m) {
                    const int bit = 31 - __clz(m);
                    m &= ~(1u << bit);
                    const uint2 q = p[(wi << 5) + bit];
                    if (__uint_as_float(q.x) < d_occ) continue;  // foreground (O2)
                    if (!f.add(q.y)) {
                        live = false;
                        break;
                    }
                }
            }
        }
        if (f.any()) return f.result();
        return pv[R].y;
    }
    if (L >= 0) return pv[L].y;
    return 0u;
}

// Per-thread record of the bulk-copy stages (every thread keeps the same copy):
// bit st of `phase` is the parity of the next wait on stage st, bit st of `pending`
// says a copy into stage st has been issued and not yet waited for.
struct StageState {
    uint32_t phase = 0;
    uint32_t pending = 0;
};

__device__ __forceinline__ void issue_row(const FrameArgs& f, const Smem& s, int wcap, int st, int row,
                                          uint32_t row_bytes)
{
    const size_t off = (size_t)row * (size_t)f.w;
    mbar_expect_tx(&s.bar[st], 2u * row_bytes);
    bulk_g2s(s.sdepth + (size_t)st * wcap, f.depth + off, row_bytes, &s.bar[st]);
    bulk_g2s(s.scolor + (size_t)st * wcap, f.color + off, row_bytes, &s.bar[st]);
}

// One band [y0, y1) of one frame.  Returns false if a bounded wait ran out.
template <int NT>
__device__ __forceinline__ bool run_band(const FrameArgs& f, int y0, int y1, const Smem& s, int wcap,
                                         StageState& ss)
{
    constexpr int NW = NT / 32;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int w = f.w, h = f.h;
    const int nwords = (w + 31) >> 5;
    const int ra = max(y0 - 1, 0), rb = min(y1, h - 1);
    const bool bulk = f.bulk != 0;
    const uint32_t row_bytes = (uint32_t)w * 4u;

    // Clear the first slot; issue the first bulk copies.
    {
        unsigned long long* k0 = s.keys + (size_t)(ra & 3) * wcap;
        for (int x = tid; x < w; x += NT) k0[x] = kEmptyKey;
        if (bulk) {
            for (int st = 0; st < kStages && ra + st <= rb; ++st) {
                if (tid == 0) issue_row(f, s, wcap, st, ra + st, row_bytes);
                ss.pending |= 1u << st;
            }
        }
    }
    __syncthreads();

    for (int r = ra; r <= rb + 1; ++r) {
        const int st = (r - ra) % kStages;
        // ---- P1: disparity and nearest-wins scatter of source row r
        if (r <= rb) {
            bool ok = true;
            if (bulk) {
                ok = mbar_wait_bounded(&s.bar[st], (ss.phase >> st) & 1u);
                if (ok) {
                    ss.phase ^= 1u << st;
                    ss.pending &= ~(1u << st);
                } else {
                    s.flag[0] = 1;
                }
            }
            if (ok) {
                unsigned long long* kr = s.keys + (size_t)(r & 3) * wcap;
                const float* drow = bulk ? s.sdepth + (size_t)st * wcap : f.depth + (size_t)r * w;
                for (int x = tid; x < w; x += NT) {
                    float zc;
                    const int xt = disparity_target(drow[x], x, f.k, f.near_, f.far_, zc);
                    if (xt >= 0 && xt < w) atomicMin(&kr[xt], zkey(zc, x));
                }
            }
        }
        __syncthreads();
        if (s.flag[0]) return false;
        // ---- P2: resolve row r in place, reached bitmask; clear the next slot
        if (r <= rb) {
            unsigned long long* kr = s.keys + (size_t)(r & 3) * wcap;
            uint32_t* br = s.bits + (size_t)(r & 3) * (wcap / 32);
            const uint32_t* crow = bulk ? s.scolor + (size_t)st * wcap : f.color + (size_t)r * w;
            for (int g = warp; g < nwords; g += NW) {
                const int x = (g << 5) + lane;
                const unsigned long long key = (x < w) ? kr[x] : kEmptyKey;
                const bool reached = key != kEmptyKey;
                const uint32_t m = __ballot_sync(0xffffffffu, reached);
                if (lane == 0) br[g] = m;
                if (reached) {
                    const uint32_t rgba = crow[(uint32_t)key];
                    reinterpret_cast<uint2*>(kr)[x] = make_uint2((uint32_t)(key >> 32), rgba);
                }
            }
            if (r + 1 <= rb) {
                unsigned long long* kn = s.keys + (size_t)((r + 1) & 3) * wcap;
                for (int x = tid; x < w; x += NT) kn[x] = kEmptyKey;
            }
        }
        __syncthreads();
        // ---- P3: fill and store row v = r - 1; refill the stage row r used
        if (bulk && r + kStages <= rb) {
            if (tid == 0) issue_row(f, s, wcap, st, r + kStages, row_bytes);
            ss.pending |= 1u << st;
        }
        const int v = r - 1;
        if (v >= y0 && v < y1) {
            const uint2* pr[3];
            const uint32_t* brow[3];
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                const int vv = v - 1 + k;
                const bool in = vv >= 0 && vv < h;
                pr[k] = in ? reinterpret_cast<const uint2*>(s.keys + (size_t)(vv & 3) * wcap) : nullptr;
                brow[k] = in ? s.bits + (size_t)(vv & 3) * (wcap / 32) : nullptr;
            }
            const uint32_t* bv = brow[1];
            const uint2* pv = pr[1];
            uint32_t* orow = f.out + (size_t)v * w;
            uint8_t* mrow = f.mask + (size_t)v * w;
            for (int b = warp; (b << 7) < w; b += NW) {
                const int xb = b << 7;
                // holes of this 128-pixel block, 4 words
                uint32_t hw[4];
                int nh = 0;
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const int g = (xb >> 5) + q;
                    const int rem = w - (g << 5);
                    const uint32_t inb = rem >= 32 ? ~0u : (rem > 0 ? ((1u << rem) - 1u) : 0u);
                    hw[q] = g < nwords ? (~bv[g] & inb) : 0u;
                    nh += __popc(hw[q]);
                }
                // fill the holes, 32 lanes at a time
                for (int base = 0; base < nh; base += 32) {
                    const int i = base + lane;
                    if (i < nh) {
                        int q = 0, c = i;
                        while (c >= __popc(hw[q])) {
                            c -= __popc(hw[q]);
                            ++q;
                        }
                        uint32_t m = hw[q];
                        for (int z = 0; z < c; ++z) m &= m - 1u;
                        const int x = xb + (q << 5) + __ffs(m) - 1;
                        s.outrow[x] = fill_pixel(x, w, nwords, pr, brow);
                    }
                }
                // reached pixels: lane owns 4 consecutive pixels
                const int x0 = xb + (lane << 2);
                uint32_t mk = 0;
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    const int x = x0 + i;
                    if (x < w) {
                        const bool reached = (bv[x >> 5] >> (x & 31)) & 1u;
                        if (reached) s.outrow[x] = pv[x].y;
                        mk |= (reached ? 0u : 1u) << (8 * i);
                    }
                }
                __syncwarp();
                if (bulk && x0 + 3 < w) {
                    const uint4 o4 = *reinterpret_cast<const uint4*>(&s.outrow[x0]);
                    *reinterpret_cast<uint4*>(orow + x0) = o4;
                    *reinterpret_cast<uint32_t*>(mrow + x0) = mk;
                } else {
#pragma unroll
                    for (int i = 0; i < 4; ++i) {
                        const int x = x0 + i;
                        if (x < w) {
                            orow[x] = s.outrow[x];
                            mrow[x] = (uint8_t)((mk >> (8 * i)) & 255u);
                        }
                    }
                }
            }
        }
    }
    __syncthreads();
    return true;
}

// After an abort, wait (bounded) for the bulk copies this CTA may still have in
// flight, so that no copy lands in shared memory after the CTA has left.
__device__ void drain_after_abort(const Smem& s, const StageState& ss, int* status)
{
    if (threadIdx.x == 0) {
        atomicExch(status, 1);
        for (int st = 0; st < kStages; ++st)
            if ((ss.pending >> st) & 1u) mbar_wait_bounded(&s.bar[st], (ss.phase >> st) & 1u);
    }
    __syncthreads();
}

template <int NT>
__global__ void __launch_bounds__(NT) fused_single(FrameArgs f, int wcap, int* status)
{
    extern __shared__ __align__(128) unsigned char smem_raw[];
    Smem s(smem_raw, wcap);
    if (threadIdx.x == 0) {
        for (int st = 0; st < kStages; ++st) mbar_init(&s.bar[st], 1);
        s.flag[0] = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    StageState ss;
    const int y0 = blockIdx.x * f.band;
    const int y1 = min(y0 + f.band, f.h);
    if (!run_band<NT>(f, y0, y1, s, wcap, ss)) drain_after_abort(s, ss, status);
}

template <int NT>
__global__ void __launch_bounds__(NT) fused_batch(const __grid_constant__ BatchArgs a, int wcap, int* status)
{
    extern __shared__ __align__(128) unsigned char smem_raw[];
    Smem s(smem_raw, wcap);
    if (threadIdx.x == 0) {
        for (int st = 0; st < kStages; ++st) mbar_init(&s.bar[st], 1);
        s.flag[0] = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    StageState ss;
    for (int item = blockIdx.x; item < a.total_items; item += gridDim.x) {
        int lo = 0, hi = a.n - 1;  // frame whose item range holds `item`
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (a.item_start[mid] <= item) lo = mid;
            else hi = mid - 1;
        }
        const FrameArgs& f = a.f[lo];
        const int y0 = (item - a.item_start[lo]) * f.band;
        const int y1 = min(y0 + f.band, f.h);
        if (!run_band<NT>(f, y0, y1, s, wcap, ss)) {
            drain_after_abort(s, ss, status);
            return;
        }
    }
}

constexpr int kThreads = 256;

}  // namespace

size_t fused_smem_bytes(int wcap)
{
    return (size_t)4 * wcap * 8 + (size_t)4 * (wcap / 32) * 4 + (size_t)wcap * 4 +
           (size_t)kStages * wcap * 8 + (size_t)kStages * 8 + 16;
}

int fused_wcap(int w) { return ((w + 127) / 128) * 128; }

int fused_threads() { return kThreads; }

cudaError_t fused_configure(int device, FusedLimits* lim)
{
    int smem_optin = 0, sms = 0, smem_sm = 0;
    cudaError_t e = cudaDeviceGetAttribute(&smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, device);
    if (e != cudaSuccess) return e;
    e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
    if (e != cudaSuccess) return e;
    e = cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, device);
    if (e != cudaSuccess) return e;
    lim->sms = sms;
    lim->smem_per_block = smem_optin;
    lim->smem_per_sm = smem_sm;
    int wmax = 0;
    while (fused_smem_bytes(wmax + 128) <= (size_t)smem_optin) wmax += 128;
    lim->max_width = wmax;
    e = cudaFuncSetAttribute(fused_single<kThreads>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_optin);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(fused_batch<kThreads>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_optin);
    return e;
}

// CTAs of `smem` bytes that fit on one SM (1 KB of each CTA's shared memory is
// reserved by the hardware).
static int ctas_per_sm(const FusedLimits& lim, size_t smem)
{
    int n = (int)((size_t)lim.smem_per_sm / (smem + 1024));
    return n < 1 ? 1 : (n > 8 ? 8 : n);
}

int fused_band_rows(const FusedLimits& lim, int w, int h)
{
    const size_t smem = fused_smem_bytes(fused_wcap(w));
    const long slots = (long)lim.sms * ctas_per_sm(lim, smem);
    int band = (int)((h + slots - 1) / slots);
    return band < 1 ? 1 : band;
}

cudaError_t fused_launch(const FrameArgs& f, const FusedLimits& lim, int* status, cudaStream_t stream)
{
    const int wcap = fused_wcap(f.w);
    const size_t smem = fused_smem_bytes(wcap);
    const int grid = (f.h + f.band - 1) / f.band;
    fused_single<kThreads><<<grid, kThreads, smem, stream>>>(f, wcap, status);
    return cudaGetLastError();
}

cudaError_t fused_launch_batch(const BatchArgs& a, int wmax, const FusedLimits& lim, int* status,
                               cudaStream_t stream)
{
    const int wcap = fused_wcap(wmax);
    const size_t smem = fused_smem_bytes(wcap);
    int grid = lim.sms * ctas_per_sm(lim, smem);
    if (grid > a.total_items) grid = a.total_items;
    if (grid < 1) return cudaSuccess;
    fused_batch<kThreads><<<grid, kThreads, smem, stream>>>(a, wcap, status);
    return cudaGetLastError();
}

}  // namespace yoro
