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

// Hole edges of pixel (v, x): L = highest reached column < x (or -1), R = lowest
// reached column > x (or w), from the row's reached bitmask.
__device__ __forceinline__ void find_edges(int x, int v, int ra, int nwords, const uint32_t* bits, int w, int& L,
                                           int& R)
{
    const uint32_t* bv = bits + (size_t)(v - ra) * nwords;
    L = -1;
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
    R = w;  // bits past the row end are zero
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
}

// Hole fill of pixel (v, x) with edges L, R (R < w).  Rows of the band are addressed
// relative to `ra`; rows outside [0, h) are skipped.  Pairs are (depth bits, rgba).
__device__ __forceinline__ uint32_t fill_from_edges(int x, int v, int L, int R, int ra, int h, int w, int nwords,
                                                    int wpad, const unsigned long long* keys, const uint32_t* bits)
{
    const uint2* pv = reinterpret_cast<const uint2*>(keys + (size_t)(v - ra) * wpad);
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

// Fill of a batch of holes, one per lane below `cnt` (none on the image border).
__device__ __forceinline__ uint32_t fill_batch(int cnt, int x, int v, int ra, int h, int w, int nwords, int wpad,
                                               const unsigned long long* keys, const uint32_t* bits)
{
    uint32_t res = 0u;
    if ((int)(threadIdx.x & 31) < cnt) {
        int L, R;
        find_edges(x, v, ra, nwords, bits, w, L, R);
        res = fill_from_edges(x, v, L, R, ra, h, w, nwords, wpad, keys, bits);
    }
    return res;
}

// Hole fill of a one-pixel crack (v, x): reached pixels at x-1 and x+1, so L = x-1,
// R = x+1, w = 2 and t = 1/2.  The kernel is rows v-1, v, v+1 times columns
// min(x+3, W-1) .. x+1; all nine slots are visited in the same order as fill_from_edges,
// without early exits.  A slot that does not contribute (outside the image, a hole, or
// nearer than the occluder) is given weight 0, which leaves acc and wrem unchanged
// exactly, so the result equals the general loop's.
__device__ __forceinline__ uint32_t fill_crack(int x, int v, int ra, int h, int w, int nwords, int wpad,
                                               const unsigned long long* keys, const uint32_t* bits)
{
    const uint2* pv = reinterpret_cast<const uint2*>(keys + (size_t)(v - ra) * wpad);
    const float d_occ = __uint_as_float(pv[x - 1].x);
    FillAcc f;
    f.init(0.5f);
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const int vv = v - 1 + k;
        const bool row_in = vv >= 0 && vv < h;
        const int j = row_in ? vv - ra : v - ra;  // a valid row to read when vv is outside
        const uint32_t* b = bits + (size_t)j * nwords;
        const uint2* p = reinterpret_cast<const uint2*>(keys + (size_t)j * wpad);
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const int col = x + 3 - c;
            const bool col_in = col < w;
            const int cc = col_in ? col : x + 1;
            const bool reached = (b[cc >> 5] >> (cc & 31)) & 1u;
            const uint2 q = p[cc];
            const bool contributes = row_in && col_in && reached && !(__uint_as_float(q.x) < d_occ);
            f.add_if(contributes, q.y);
        }
    }
    return f.any() ? f.result() : pv[x + 1].y;
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
                                         unsigned long long* keys, uint32_t* bits, int* ctr, int* lastr)
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
        if (tid == 0) *ctr = 0;
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
                    if (lane == 0) bits[(size_t)(j0 + u) * nwords + g] = m;
                    if (reached)
                        reinterpret_cast<uint2*>(keys + (size_t)(j0 + u) * wpad)[x] = make_uint2(kp[u].y, rgba[u]);
                }
            }
        }
    }
    __syncthreads();

    // Last reached column of every band row: holes right of it have no background edge
    // (R = W) and take the fallback, the color of that last reached pixel (zero if the row
    // has none).  They leave with the reached pixels; the fill below skips them.
    for (int vj = warp; vj < y1 - y0; vj += NW) {
        const uint32_t* bv = bits + (size_t)(vj + y0 - ra) * nwords;
        int last = -1;
        for (int g = lane; g < nwords; g += 32)
            if (bv[g]) last = (g << 5) + 31 - __clz(bv[g]);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) last = max(last, __shfl_xor_sync(0xffffffffu, last, o));
        if (lane == 0) lastr[vj] = last;
    }
    __syncthreads();

    // ---- P3a: reached pixels, border holes and the hole mask leave
    for (int v = y0; v < y1; ++v) {
        const int j = v - ra;
        const uint32_t* bv = bits + (size_t)j * nwords;
        const uint2* pv = reinterpret_cast<const uint2*>(keys + (size_t)j * wpad);
        const int last = lastr[v - y0];
        const uint32_t border = last >= 0 ? pv[last].y : 0u;
        uint32_t* orow = f.out + (size_t)v * w;
        uint8_t* mrow = f.mask + (size_t)v * w;
        for (int x0 = tid << 2; x0 < w; x0 += NT * 4) {
            const uint32_t nib = (bv[x0 >> 5] >> (x0 & 31)) & 15u;  // reached flags of x0..x0+3
            if (f.bulk && x0 + 3 < w) {
                const uint4 p01 = *reinterpret_cast<const uint4*>(pv + x0);
                const uint4 p23 = *reinterpret_cast<const uint4*>(pv + x0 + 2);
                uint4 o = make_uint4(p01.y, p01.w, p23.y, p23.w);
                if (x0 + 0 > last) o.x = border;
                if (x0 + 1 > last) o.y = border;
                if (x0 + 2 > last) o.z = border;
                if (x0 + 3 > last) o.w = border;
                // bytes of interior holes are left to the fill
                const uint32_t wr = nib | (x0 + 0 > last ? 1u : 0u) | (x0 + 1 > last ? 2u : 0u) |
                                    (x0 + 2 > last ? 4u : 0u) | (x0 + 3 > last ? 8u : 0u);
                if (wr == 15u) {
                    *reinterpret_cast<uint4*>(orow + x0) = o;
                } else {
                    if (wr & 1u) orow[x0] = o.x;
                    if (wr & 2u) orow[x0 + 1] = o.y;
                    if (wr & 4u) orow[x0 + 2] = o.z;
                    if (wr & 8u) orow[x0 + 3] = o.w;
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
                        else if (x > last) orow[x] = border;
                        mrow[x] = reached ? 0 : 1;
                    }
                }
            }
        }
    }

    // ---- P3b: fill of the interior holes.  Work units are segments of kSeg words of a
    // band row, taken by warps from a shared counter, so that busy rows spread over the
    // warps while the holes of one disocclusion stay together.  A warp reads one word per
    // lane and packs one-pixel cracks and wider holes into two separate batches of up to
    // 32, one hole per lane, so that the lanes of a batch run the same code.
    {
        constexpr int kSeg = 8;
        const int nseg = (nwords + kSeg - 1) / kSeg;
        const int nunits = (y1 - y0) * nseg;
        int cx = 0, cv = 0, ccnt = 0;  // crack batch: this lane's pixel, batch size
        int gx = 0, gv = 0, gcnt = 0;  // general batch
        for (;;) {
            int unit = 0;
            if (lane == 0) unit = atomicAdd(ctr, 1);
            unit = __shfl_sync(0xffffffffu, unit, 0);
            if (unit >= nunits) break;
            const int vj = unit / nseg;
            const int g0 = (unit - vj * nseg) * kSeg;
            const int v = y0 + vj;
            const uint32_t* bv = bits + (size_t)(v - ra) * nwords;
            const int last = lastr[vj];
            const int g = g0 + lane;
            const bool gin = lane < kSeg && g < nwords;
            const uint32_t reach = gin ? bv[g] : 0u;
            // interior holes: columns up to the last reached one
            const int rem = last - (g << 5);
            const uint32_t inb = rem >= 31 ? ~0u : (rem >= 0 ? ((2u << rem) - 1u) : 0u);
            const uint32_t hw = gin ? (~reach & inb) : 0u;
            // neighbour words for the crack test (the lanes beside, or memory at the segment ends)
            uint32_t prev = __shfl_up_sync(0xffffffffu, reach, 1);
            uint32_t next = __shfl_down_sync(0xffffffffu, reach, 1);
            if (lane == 0) prev = g > 0 ? bv[g - 1] : 0u;
            if (lane == kSeg - 1 || g + 1 >= nwords) next = (gin && g + 1 < nwords) ? bv[g + 1] : 0u;
            const uint32_t left = (reach << 1) | (prev >> 31);   // bit i: column 32g + i - 1 reached
            const uint32_t right = (reach >> 1) | (next << 31);  // bit i: column 32g + i + 1 reached
            const uint32_t cm_l = hw & left & right;
            const uint32_t gm_l = hw & ~cm_l;
            uint32_t words = __ballot_sync(0xffffffffu, hw != 0u);
            while (words) {
                const int sl = __ffs(words) - 1;
                words &= words - 1u;
                const uint32_t cm = __shfl_sync(0xffffffffu, cm_l, sl);
                const uint32_t gm = __shfl_sync(0xffffffffu, gm_l, sl);
                const int wg = g0 + sl;
                const int nc = __popc(cm), ng = __popc(gm);
                if (ccnt + nc > 32) {
                    if (lane < ccnt)
                        f.out[(size_t)cv * w + cx] = fill_crack(cx, cv, ra, h, w, nwords, wpad, keys, bits);
                    ccnt = 0;
                }
                if (gcnt + ng > 32) {
                    const uint32_t o = fill_batch(gcnt, gx, gv, ra, h, w, nwords, wpad, keys, bits);
                    if (lane < gcnt) f.out[(size_t)gv * w + gx] = o;
                    gcnt = 0;
                }
                const int kc = lane - ccnt, kg = lane - gcnt;
                if (kc >= 0 && kc < nc) {
                    cx = (wg << 5) + nth_set_bit(cm, kc);
                    cv = v;
                }
                if (kg >= 0 && kg < ng) {
                    gx = (wg << 5) + nth_set_bit(gm, kg);
                    gv = v;
                }
                ccnt += nc;
                gcnt += ng;
            }
        }
        if (lane < ccnt) f.out[(size_t)cv * w + cx] = fill_crack(cx, cv, ra, h, w, nwords, wpad, keys, bits);
        {
            const uint32_t o = fill_batch(gcnt, gx, gv, ra, h, w, nwords, wpad, keys, bits);
            if (lane < gcnt) f.out[(size_t)gv * w + gx] = o;
        }
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
    int* ctr = reinterpret_cast<int*>(bits + (size_t)slots * ((wpad + 31) / 32));
    int* lastr = ctr + 4;
    const int nbands = (f.h + f.band - 1) / f.band;
    for (int b = blockIdx.x; b < nbands; b += gridDim.x) {
        const int y0 = b * f.band;
        run_band<NT>(f, y0, min(y0 + f.band, f.h), wpad, keys, bits, ctr, lastr);
    }
}

template <int NT, int MINB>
__global__ void __launch_bounds__(NT, MINB) fused_batch(const __grid_constant__ BatchArgs a, int wpad)
{
    extern __shared__ __align__(128) unsigned char smem_raw[];
    const int slots = a.max_band + 2;
    unsigned long long* keys = reinterpret_cast<unsigned long long*>(smem_raw);
    uint32_t* bits = reinterpret_cast<uint32_t*>(smem_raw + (size_t)slots * wpad * 8);
    int* ctr = reinterpret_cast<int*>(bits + (size_t)slots * ((wpad + 31) / 32));
    int* lastr = ctr + 4;
    for (int item = blockIdx.x; item < a.total_items; item += gridDim.x) {
        int lo = 0, hi = a.n - 1;  // frame whose item range holds `item`
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (a.item_start[mid] <= item) lo = mid;
            else hi = mid - 1;
        }
        const FrameArgs& f = a.f[lo];
        const int y0 = (item - a.item_start[lo]) * f.band;
        run_band<NT>(f, y0, min(y0 + f.band, f.h), wpad, keys, bits, ctr, lastr);
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
    // keys, reached bitmasks, a work counter (16 bytes) and the last reached column of
    // each band row
    return slots * (size_t)wpad * 8 + slots * (size_t)((wpad + 31) / 32) * 4 + 16 + (size_t)band * 4;
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
    // One CTA per (frame, band) item: the hardware block scheduler hands the next item to
    // whichever SM frees up first, so bands with heavy disocclusions do not hold back the
    // rest of the batch.
    const int grid = a.total_items;
    if (grid < 1) return cudaSuccess;
    if (two)
        fused_batch<kSmall, 2><<<grid, kSmall, smem, stream>>>(a, wpad);
    else
        fused_batch<kBig, 1><<<grid, kBig, smem, stream>>>(a, wpad);
    return cudaGetLastError();
}

int fused_max_band(const FusedLimits& lim, int w) { return max_band(lim, fused_wpad(w)); }

}  // namespace yoro
