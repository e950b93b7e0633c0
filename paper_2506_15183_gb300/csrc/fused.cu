// Fused second-eye synthesis kernel for GB300 (sm_103a).
//
// One CTA synthesizes a band of B output rows at once; shared memory holds the
// band's warped rows plus one halo row above and below (rows y0-1 .. y0+B), each as
// 64-bit z-buffer keys that become (depth, RGBA8) pairs.  Four steps, three CTA
// barriers per band:
//
//   0.  one thread starts 1-D bulk prefetches of the band's depth and color rows
//       into L2 (cp.async.bulk.prefetch.L2), while all threads clear the keys;
//   P1  disparity + forward warp (Alg. 1 closed form, Alg. 2 nearest kept): every
//       source pixel of every row does a 64-bit atomicMin of
//       (depth bits << 32 | source column) into its row's keys (O1: a row never
//       writes another row);
//   P2  resolve + gather: each key becomes (depth, RGBA8 of its source) in place;
//       warp ballots write the rows' reached-pixel bitmasks;
//   P3  the band's rows leave: reached pixels and the hole mask by 16-byte / 4-byte
//       stores; holes are filled (Alg. 3, Eq. 6) by warps that take the band's
//       32-pixel words round-robin, one hole per lane, so a wide disocclusion is
//       spread over many warps.  Hole edges and kernel candidates come from the
//       bitmasks (leading/trailing-zero counts over 32-pixel words).
//
// No thread ever waits on another CTA or on an asynchronous copy: the prefetches
// only warm L2, and every read is an ordinary load.
#include <cuda_runtime.h>

#include <cstdint>

#include "yoro_device.cuh"
#include "yoro_internal.h"

namespace yoro {

namespace {

constexpr float kSettleFrom = 0.0009765625f;  // 2^-10: start testing the exact early exit

__device__ __forceinline__ void prefetch_l2(const void* p, uint32_t bytes)
{
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p), "r"(bytes) : "memory");
}

// Hole fill of pixel (v, x).  `keys`/`bits` point at the slot of row `ra`; rows
// outside [0, h) are skipped.  Pairs are (depth bits, rgba) per reached column.
__device__ __forceinline__ uint32_t fill_pixel(int x, int v, int ra, int h, int w, int nwords, int wpad,
                                               const unsigned long long* keys, const uint32_t* bits)
{
    const int jv = v - ra;
    const uint32_t* bv = bits + (size_t)jv * nwords;
    const uint2* pv = reinterpret_cast<const uint2*>(keys + (size_t)jv * wpad);
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
    if (R >= w) return (L >= 0) ? pv[L].y : 0u;
    const int wd = R - L;
    const float d_occ = (L >= 0) ? __uint_as_float(pv[L].x) : 0.0f;
    FillAcc f;
    f.init(__fdiv_rn((float)(R - x), (float)wd));
    const int jhi = min(R + wd, w - 1);
    const int whi = jhi >> 5, wlo = R >> 5;
    const uint32_t mhi = ((jhi & 31) == 31) ? ~0u : ((2u << (jhi & 31)) - 1u);
    const uint32_t mlo = ~0u << (R & 31);
#pragma unroll 1
    for (int vv = v - 1; vv <= v + 1; ++vv) {
        if (vv < 0 || vv >= h) continue;
        const uint32_t* b = bits + (size_t)(vv - ra) * nwords;
        const uint2* p = reinterpret_cast<const uint2*>(keys + (size_t)(vv - ra) * wpad);
#pragma unroll 1
        for (int wi = whi; wi >= wlo; --wi) {
            uint32_t m = b[wi];
            if (wi == whi) m &= mhi;
            if (wi == wlo) m &= mlo;
            while (m) {
                const int bit = 31 - __clz(m);
                m &= ~(1u << bit);
                const uint2 q = p[(wi << 5) + bit];
                if (__uint_as_float(q.x) < d_occ) continue;  // foreground (O2)
                if (!f.add(q.y)) return f.result();          // weight reached exactly 0
                uint32_t out;
                if (f.wrem <= kSettleFrom && f.settled(out)) return out;
            }
        }
    }
    return f.any() ? f.result() : pv[R].y;
}

// Position of the k-th (0-based) set bit of m; m must have more than k set bits.
__device__ __forceinline__ int nth_set_bit(uint32_t m, int k)
{
    int pos = 0, c;
    c = __popc(m & 0xffffu);
    if (k >= c) { k -= c; pos += 16; m >>= 16; }
    c = __popc(m & 0xffu);
    if (k >= c) { k -= c; pos += 8; m >>= 8; }
    c = __popc(m & 0xfu);
    if (k >= c) { k -= c; pos += 4; m >>= 4; }
    c = __popc(m & 0x3u);
    if (k >= c) { k -= c; pos += 2; m >>= 2; }
    c = (int)(m & 1u);
    if (k >= c) pos += 1;
    return pos;
}

// One band [y0, y1) of one frame; shared memory holds rows ra..rb (ra = y0-1 or 0,
// rb = y1 or h-1), row j at keys + j*wpad and bits + j*nwords.  Warp `warp` owns the
// 32-pixel columns x = warp*32 + lane (+ NT, + 2*NT, ...) of every row in P1 and P2.
// Ends with a barrier, so the next band may reuse shared memory.
template <int NT>
__device__ __forceinline__ void run_band(const FrameArgs& f, int y0, int y1, int wpad,
                                         unsigned long long* keys, uint32_t* bits, uint32_t* hword)
{
    constexpr int NW = NT / 32;
    constexpr int RB = 8;  // rows per batch of loads
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int w = f.w, h = f.h;
    const int nwords = (w + 31) >> 5;
    const int ra = max(y0 - 1, 0), rb = min(y1, h - 1);
    const int nr = rb - ra + 1;
    const float* depth = f.depth + (size_t)ra * w;
    const uint32_t* color = f.color + (size_t)ra * w;

    if (f.bulk && warp == 0) {  // depth first: P1 needs it before P2 needs color
        for (int j = lane; j < nr; j += 32) prefetch_l2(depth + (size_t)j * w, (uint32_t)w * 4u);
        for (int j = lane; j < nr; j += 32) prefetch_l2(color + (size_t)j * w, (uint32_t)w * 4u);
    }
    {
        uint4* k4 = reinterpret_cast<uint4*>(keys);  // two keys per 16 bytes; wpad % 8 == 0
        const int n4 = nr * (wpad >> 1);
        const uint4 e = make_uint4(~0u, ~0u, ~0u, ~0u);
        for (int i = tid; i < n4; i += NT) k4[i] = e;
        const int nhw = ((y1 - y0) * nwords + 31) >> 5;
        for (int i = tid; i < nhw; i += NT) hword[i] = 0u;
    }
    __syncthreads();

    // ---- P1: disparity and nearest-wins scatter of rows ra..rb
    for (int g = warp; g < nwords; g += NW) {
        const int x = (g << 5) + lane;
        const bool xin = x < w;
        const float xc = __fadd_rn((float)x, 0.5f);
        for (int j0 = 0; j0 < nr; j0 += RB) {
            float z[RB];
#pragma unroll
            for (int u = 0; u < RB; ++u)
                z[u] = (xin && j0 + u < nr) ? __ldg(depth + (size_t)(j0 + u) * w + x) : 0.0f;
#pragma unroll
            for (int u = 0; u < RB; ++u) {
                if (xin && j0 + u < nr) {
                    float zc;
                    const int xt = disparity_target(z[u], xc, f.k, f.near_, f.far_, f.half_m, zc);
                    if ((unsigned)xt < (unsigned)w) atomicMin(&keys[(size_t)(j0 + u) * wpad + xt], zkey(zc, x));
                }
            }
        }
    }
    __syncthreads();

    // ---- P2: resolve in place, gather colors, reached bitmasks
    for (int g = warp; g < nwords; g += NW) {
        const int x = (g << 5) + lane;
        const bool xin = x < w;
        for (int j0 = 0; j0 < nr; j0 += RB) {
            uint2 kp[RB];  // (source column, depth bits) of each key
            uint32_t rgba[RB];
#pragma unroll
            for (int u = 0; u < RB; ++u)
                kp[u] = (xin && j0 + u < nr) ? reinterpret_cast<const uint2*>(keys + (size_t)(j0 + u) * wpad)[x]
                                             : make_uint2(~0u, ~0u);
#pragma unroll
            for (int u = 0; u < RB; ++u)  // a key's high word is ~0 only while empty
                rgba[u] = (kp[u].y != ~0u) ? __ldg(color + (size_t)(j0 + u) * w + kp[u].x) : 0u;
#pragma unroll
            for (int u = 0; u < RB; ++u) {
                if (j0 + u < nr) {  // warp-uniform
                    const bool reached = kp[u].y != ~0u;
                    const uint32_t m = __ballot_sync(0xffffffffu, reached);
                    if (lane == 0) {
                        bits[(size_t)(j0 + u) * nwords + g] = m;
                        const int vb = j0 + u + ra - y0;  // row within the band, or a halo row
                        const int rem = w - (g << 5);
                        const uint32_t inb = rem >= 32 ? ~0u : ((1u << rem) - 1u);
                        if (vb >= 0 && vb < y1 - y0 && (~m & inb)) {
                            const int q = vb * nwords + g;
                            atomicOr(&hword[q >> 5], 1u << (q & 31));
                        }
                    }
                    if (reached)
                        reinterpret_cast<uint2*>(keys + (size_t)(j0 + u) * wpad)[x] = make_uint2(kp[u].y, rgba[u]);
                }
            }
        }
    }
    __syncthreads();

    // ---- P3a: reached pixels and the hole mask leave
    for (int v = y0; v < y1; ++v) {
        const int j = v - ra;
        const uint32_t* bv = bits + (size_t)j * nwords;
        const uint2* pv = reinterpret_cast<const uint2*>(keys + (size_t)j * wpad);
        uint32_t* orow = f.out + (size_t)v * w;
        uint8_t* mrow = f.mask + (size_t)v * w;
        for (int x0 = tid << 2; x0 < w; x0 += NT * 4) {
            const uint32_t nib = (bv[x0 >> 5] >> (x0 & 31)) & 15u;  // reached flags of x0..x0+3
            if (f.bulk && x0 + 3 < w) {
                const uint4 p01 = *reinterpret_cast<const uint4*>(pv + x0);
                const uint4 p23 = *reinterpret_cast<const uint4*>(pv + x0 + 2);
                if (nib == 15u) {
                    *reinterpret_cast<uint4*>(orow + x0) = make_uint4(p01.y, p01.w, p23.y, p23.w);
                } else {
                    if (nib & 1u) orow[x0] = p01.y;
                    if (nib & 2u) orow[x0 + 1] = p01.w;
                    if (nib & 4u) orow[x0 + 2] = p23.y;
                    if (nib & 8u) orow[x0 + 3] = p23.w;
                }
                const uint32_t hn = ~nib & 15u;
                *reinterpret_cast<uint32_t*>(mrow + x0) =
                    (hn & 1u) | ((hn & 2u) << 7) | ((hn & 4u) << 14) | ((hn & 8u) << 21);
            } else {
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    const int x = x0 + i;
                    if (x < w) {
                        const bool reached = (nib >> i) & 1u;
                        if (reached) orow[x] = pv[x].y;
                        mrow[x] = reached ? 0 : 1;
                    }
                }
            }
        }
    }

    // ---- P3b: hole fill.  The band's words that hold holes (flags in `hword`, in
    // row-major order) are split into NW equal ranges of consecutive words, one per
    // warp, so neighbouring holes of one disocclusion go to the same warp and run the
    // same candidate sequence.  A warp packs the holes of its words into batches of up
    // to 32, one hole per lane.
    {
        const int nhw = ((y1 - y0) * nwords + 31) >> 5;
        // lane L counts the flagged words among hword[L], hword[L + 32], ...
        int mine = 0;
        for (int i = lane; i < nhw; i += 32) mine += __popc(hword[i]);
        int total = mine;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) total += __shfl_xor_sync(0xffffffffu, total, o);
        const int r0 = (int)(((long long)total * warp) / NW), r1 = (int)(((long long)total * (warp + 1)) / NW);
        int hx = 0, hv = 0, cnt = 0;  // this lane's hole of the current batch, batch size
        int base = 0;                 // flagged words before hword[i0 .. i0 + 31]
        for (int i0 = 0; i0 < nhw && base < r1; i0 += 32) {
            const uint32_t fw = (i0 + lane < nhw) ? hword[i0 + lane] : 0u;
            const int c = __popc(fw);
            int incl = c;  // inclusive prefix over lanes
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int t = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += t;
            }
            const int excl = base + incl - c;
            const int seg_total = __shfl_sync(0xffffffffu, incl, 31);
            // this lane's flags have ranks excl .. excl + c - 1 (lowest bit first); keep
            // those with rank in [r0, r1)
            uint32_t sel = 0u;
            {
                const int first = max(r0, excl), last = min(r1, excl + c);
                if (first < last) {
                    sel = fw;
                    for (int z = excl; z < first; ++z) sel &= sel - 1u;  // drop ranks below r0
                    uint32_t rest = sel;                                 // drop ranks from r1 on
                    for (int z = first; z < last; ++z) rest &= rest - 1u;
                    sel &= ~rest;
                }
            }
            uint32_t lanes = __ballot_sync(0xffffffffu, sel != 0u);
            while (lanes) {
                const int sl = __ffs(lanes) - 1;
                lanes &= lanes - 1u;
                uint32_t words = __shfl_sync(0xffffffffu, sel, sl);
                while (words) {
                    const int q = ((i0 + sl) << 5) + __ffs(words) - 1;
                    words &= words - 1u;
                    const int vj = q / nwords, g = q - vj * nwords;
                    const int v = y0 + vj;
                    const int rem = w - (g << 5);
                    const uint32_t inb = rem >= 32 ? ~0u : ((1u << rem) - 1u);
                    const uint32_t wm = ~bits[(size_t)(v - ra) * nwords + g] & inb;
                    const int n = __popc(wm);
                    if (cnt + n > 32) {  // flush the full batch
                        if (lane < cnt)
                            f.out[(size_t)hv * w + hx] = fill_pixel(hx, hv, ra, h, w, nwords, wpad, keys, bits);
                        cnt = 0;
                    }
                    const int k = lane - cnt;
                    if (k >= 0 && k < n) {
                        hx = (g << 5) + nth_set_bit(wm, k);
                        hv = v;
                    }
                    cnt += n;
                }
            }
            base += seg_total;
        }
        if (lane < cnt) f.out[(size_t)hv * w + hx] = fill_pixel(hx, hv, ra, h, w, nwords, wpad, keys, bits);
    }
    __syncthreads();
}

template <int NT, int MINB>
__global__ void __launch_bounds__(NT, MINB) fused_single(FrameArgs f, int wpad)
{
    extern __shared__ __align__(128) unsigned char smem_raw[];
    const int slots = f.band + 2;
    unsigned long long* keys = reinterpret_cast<unsigned long long*>(smem_raw);
    uint32_t* bits = reinterpret_cast<uint32_t*>(smem_raw + (size_t)slots * wpad * 8);
    uint32_t* hword = bits + (size_t)slots * ((wpad + 31) / 32);
    const int nbands = (f.h + f.band - 1) / f.band;
    for (int b = blockIdx.x; b < nbands; b += gridDim.x) {
        const int y0 = b * f.band;
        run_band<NT>(f, y0, min(y0 + f.band, f.h), wpad, keys, bits, hword);
    }
}

template <int NT, int MINB>
__global__ void __launch_bounds__(NT, MINB) fused_batch(const __grid_constant__ BatchArgs a, int wpad)
{
    extern __shared__ __align__(128) unsigned char smem_raw[];
    const int slots = a.max_band + 2;
    unsigned long long* keys = reinterpret_cast<unsigned long long*>(smem_raw);
    uint32_t* bits = reinterpret_cast<uint32_t*>(smem_raw + (size_t)slots * wpad * 8);
    uint32_t* hword = bits + (size_t)slots * ((wpad + 31) / 32);
    for (int item = blockIdx.x; item < a.total_items; item += gridDim.x) {
        int lo = 0, hi = a.n - 1;  // frame whose item range holds `item`
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (a.item_start[mid] <= item) lo = mid;
            else hi = mid - 1;
        }
        const FrameArgs& f = a.f[lo];
        const int y0 = (item - a.item_start[lo]) * f.band;
        run_band<NT>(f, y0, min(y0 + f.band, f.h), wpad, keys, bits, hword);
    }
}

// Two shapes: 1024 threads with one CTA per SM (large bands), or 512 threads with
// two CTAs per SM (bands small enough that two fit in shared memory).
constexpr int kBig = 1024;
constexpr int kSmall = 512;

}  // namespace

int fused_wpad(int w) { return ((w + 7) / 8) * 8; }

size_t fused_smem_bytes(int wpad, int band)
{
    const size_t slots = (size_t)band + 2;
    // keys, reached bitmasks, and one flag bit per 32-pixel word of the band
    return slots * (size_t)wpad * 8 + slots * (size_t)((wpad + 31) / 32) * 4 +
           (((size_t)band * (size_t)((wpad + 31) / 32) + 31) / 32) * 4;
}

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
    int wmax = 0;  // widest frame with a band of one row
    while (fused_smem_bytes(fused_wpad(wmax + 32), 1) <= (size_t)smem_optin && wmax + 32 <= 65535) wmax += 32;
    lim->max_width = wmax;
    const void* fns[] = {(const void*)fused_single<kBig, 1>, (const void*)fused_single<kSmall, 2>,
                         (const void*)fused_batch<kBig, 1>, (const void*)fused_batch<kSmall, 2>};
    for (const void* fn : fns) {
        e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_optin);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

// Largest band whose rows fit the per-CTA shared memory.
static int max_band(const FusedLimits& lim, int wpad)
{
    if (wpad <= 0) return 1;
    int b = 1;
    while (b < 4096 && fused_smem_bytes(wpad, b + 1) <= (size_t)lim.smem_per_block) ++b;
    return b;
}

// Band height for a w x h frame: enough bands for every SM, each as tall as shared
// memory allows up to that.  Two CTAs per SM when two such bands fit on an SM.
FusedShape fused_shape(const FusedLimits& lim, int w, int h)
{
    const int wpad = fused_wpad(w);
    const int bmax = max_band(lim, wpad);
    FusedShape s;
    int band = (h + lim.sms - 1) / lim.sms;
    if (band > bmax) band = bmax;
    if (band < 1) band = 1;
    // two CTAs of half the band height, if they fit beside each other
    const int half = (band + 1) / 2;
    if (band >= 2 && 2 * (fused_smem_bytes(wpad, half) + 1024) <= (size_t)lim.smem_per_sm) {
        s.band = half;
        s.two_per_sm = 1;
    } else {
        s.band = band;
        s.two_per_sm = 0;
    }
    return s;
}

cudaError_t fused_launch(const FrameArgs& f, const FusedLimits& lim, int two_per_sm, cudaStream_t stream)
{
    const int wpad = fused_wpad(f.w);
    const size_t smem = fused_smem_bytes(wpad, f.band);
    const int nbands = (f.h + f.band - 1) / f.band;
    const int slots = lim.sms * (two_per_sm ? 2 : 1);
    const int grid = nbands < slots ? nbands : slots;
    if (two_per_sm)
        fused_single<kSmall, 2><<<grid, kSmall, smem, stream>>>(f, wpad);
    else
        fused_single<kBig, 1><<<grid, kBig, smem, stream>>>(f, wpad);
    return cudaGetLastError();
}

cudaError_t fused_launch_batch(const BatchArgs& a, int wmax, const FusedLimits& lim, cudaStream_t stream)
{
    const int wpad = fused_wpad(wmax);
    const size_t smem = fused_smem_bytes(wpad, a.max_band);
    const bool two = 2 * (smem + 1024) <= (size_t)lim.smem_per_sm;
    int grid = lim.sms * (two ? 2 : 1);
    if (grid > a.total_items) grid = a.total_items;
    if (grid < 1) return cudaSuccess;
    if (two)
        fused_batch<kSmall, 2><<<grid, kSmall, smem, stream>>>(a, wpad);
    else
        fused_batch<kBig, 1><<<grid, kBig, smem, stream>>>(a, wpad);
    return cudaGetLastError();
}

int fused_max_band(const FusedLimits& lim, int w) { return max_band(lim, fused_wpad(w)); }

}  // namespace yoro
