// Fused second-eye synthesis kernel for GB300 (sm_103a).
//
// One CTA synthesizes a band of B output rows at once; shared memory holds the
// band's warped rows plus the kernel's halo rows above and below (the window; one halo
// row per side for the paper's 3-row kernel): per target pixel a 32-bit word that is
// first the source column and then the depth, a 32-bit RGBA8 word, a reached bit, and
// per 32-pixel word a hole prefix sum.  The steps, separated by CTA barriers:
//
//   0.  one warp starts 1-D bulk prefetches of the window's depth and color rows
//       into L2 (cp.async.bulk.prefetch.L2), while all threads clear the window;
//   P1  disparity + forward warp (Alg. 1 closed form, Alg. 2 nearest kept): every
//       source pixel of every window row takes the atomic maximum of its source
//       column into its target's word (O1: a row never writes another row).  In a
//       row, of two sources that reach the same target the one further right is
//       the nearer (see scatter_window), so the maximum column is the z-test's
//       winner.  A thread takes whole columns (two, five rows of each per load
//       group) where they split evenly over the threads, else pixels round-robin;
//   P2  resolve + gather: each reached target loads its source's depth and color;
//       warp ballots write the rows' reached-pixel bitmasks, and the band rows'
//       reached pixels and hole mask leave for global memory at once;
//   P3a per band row: its last reached pixel, the border holes right of it (the
//       fallback), and per word the counts of cracks and wider holes with prefix sums;
//   P3b the other holes are filled (Alg. 3, Eq. 6) in chunks dealt to whichever warp
//       is free (32 pixels of wider holes, one per lane, or 64 one-pixel cracks, two
//       per lane), so a wide disocclusion is spread over many warps; a chunk inside
//       one hole is filled by the whole warp together.  Hole
//       edges and kernel candidates come from the bitmasks (leading/trailing-zero
//       counts over 32-pixel words).
//
// No thread ever waits on another CTA or on an asynchronous copy: the prefetches
// only warm L2, and every read is an ordinary load.
#include <cuda_runtime.h>

#include <cstdint>

#include "yoro_device.cuh"
#include "yoro_internal.h"

namespace yoro {

namespace {

#ifdef YORO_DEBUG_BOUNDS
__device__ unsigned g_status;  // debug-bounds status word of this file's kernels
__device__ __forceinline__ void yoro_status_record(unsigned code) { atomicOr(&g_status, code); }
#endif

// Records kSelfTest in the debug-bounds build (no memory is touched); nothing otherwise.
__global__ void selftest_kernel()
{
    if (threadIdx.x == 0) (void)YORO_BOUND(false, kSelfTest);
}

// Remaining weight below which the exact early exit is tested after each contribution
// (2^-9: measured fastest among 2^-8 .. 2^-15 on the 1832x1920 workload).
constexpr float kSettleFrom = 0.001953125f;

__device__ __forceinline__ void prefetch_l2(const void* p, uint32_t bytes)
{
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p), "r"(bytes) : "memory");
}

// The band window in shared memory.  Window row j (frame row ra + j) has its words at
// zt + j*wpad (source column during P1, -1 for none; clamped depth bits of the source
// after P2), rgba + j*wpad (color of the source after P2) and its reached bitmask at
// bits + j*nwords.
struct Window {
    uint32_t* zt;
    uint32_t* rgba;
    uint32_t* bits;
    uint32_t* pre;  // band row vj's hole prefix sums per word at pre + vj*nwords
    int wpad, nwords, ra, slots;
    __device__ __forceinline__ const uint32_t* zrow(int v) const { return zt + (v - ra) * wpad; }
    __device__ __forceinline__ const uint32_t* crow(int v) const { return rgba + (v - ra) * wpad; }
    __device__ __forceinline__ const uint32_t* brow(int v) const { return bits + (v - ra) * nwords; }
};

// The Patcher's kernel shape (Sec. Patcher): rows v - halo .. v + halo (the kernel
// height h = 2 halo + 1, the paper's default 3) and the column order in each row:
// farthest first, min(R + w, W - 1) down to R (the paper's order, mirrored), or nearest
// first, R up.  VAR = false compiles the paper's defaults as constants; VAR = true
// takes them from the frame (the variant launch).
template <bool VAR>
struct KernelShape {
    int halo;
    bool nearest;
    __device__ __forceinline__ explicit KernelShape(const FrameArgs& f)
        : halo(VAR ? f.halo : 1), nearest(VAR ? f.nearest != 0 : false)
    {
    }
};

// Hole edges of pixel (v, x): L = highest reached column < x (or -1), R = lowest
// reached column > x (or w), from the row's reached bitmask.
__device__ __forceinline__ void find_edges(int x, int v, const Window& s, int w, int& L, int& R)
{
    const uint32_t* bv = s.brow(v);
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
            if (++wi >= s.nwords) break;
            m = bv[wi];
        }
    }
}

// Hole fill of pixel (v, x) with edges L, R (R < w).  Rows outside [0, h) are skipped.
template <bool VAR>
__device__ __forceinline__ uint32_t fill_from_edges(int x, int v, int L, int R, int h, int w, const Window& s,
                                                    const KernelShape<VAR>& ks)
{
    const int wd = R - L;
    const float d_occ = (L >= 0) ? __uint_as_float(s.zrow(v)[L]) : 0.0f;
    FillAcc f;
    f.init(__fdiv_rn((float)(R - x), (float)wd));
    const int jhi = min(R + wd, w - 1);
    const int whi = jhi >> 5, wlo = R >> 5;
    const uint32_t mhi = ((jhi & 31) == 31) ? ~0u : ((2u << (jhi & 31)) - 1u);
    const uint32_t mlo = ~0u << (R & 31);
#pragma unroll 1
    for (int vv = v - ks.halo; vv <= v + ks.halo; ++vv) {
        if (vv < 0 || vv >= h || !YORO_BOUND(vv - s.ra >= 0 && vv - s.ra < s.slots, kBadHoles)) continue;
        const uint32_t* b = s.brow(vv);
        const uint32_t* zr = s.zrow(vv);
        const uint32_t* cr = s.crow(vv);
#pragma unroll 1
        for (int step = 0; step <= whi - wlo; ++step) {
            const int wi = ks.nearest ? wlo + step : whi - step;
            uint32_t m = b[wi];
            if (wi == whi) m &= mhi;
            if (wi == wlo) m &= mlo;
            while (m) {
                const int bit = ks.nearest ? __ffs(m) - 1 : 31 - __clz(m);
                m &= ~(1u << bit);
                const int c = (wi << 5) + bit;
                if (__uint_as_float(zr[c]) < d_occ) continue;  // foreground (O2)
                if (!f.add(cr[c])) return f.result();          // weight reached exactly 0
                uint32_t out;
                if (f.wrem <= kSettleFrom && f.settled(out)) return out;
            }
        }
    }
    return f.any() ? f.result() : s.crow(v)[R];
}

// Hole fill of the pixels x of one hole (row v, edges L, R with R < w), one per active
// lane, by the whole warp.  The depth gate and the candidates are the same for every
// pixel of the hole, so the warp tests 32 kernel columns at a time (ballot of the
// contributing ones) and hands each contributor's color, in Alg. 3's order, to all
// lanes; each lane accumulates it with its own t and stops at its own exact exit.  A
// kernel full of foreground candidates is thus crossed 32 columns per step instead of
// one candidate per step.
template <bool VAR>
__device__ __forceinline__ uint32_t fill_hole_warp(int x, bool act, int v, int L, int R, int h, int w,
                                                   const Window& s, const KernelShape<VAR>& ks)
{
    const int lane = threadIdx.x & 31;
    const int wd = R - L;
    const float d_occ = (L >= 0) ? __uint_as_float(s.zrow(v)[L]) : 0.0f;
    FillAcc f;
    f.init(__fdiv_rn((float)(R - (act ? x : L + 1)), (float)wd));
    bool done = !act;
    uint32_t res = 0u;
    const int jhi = min(R + wd, w - 1);
    const int jlast = min(v + ks.halo, h - 1) - s.ra;
    for (int j = max(v - ks.halo, 0) - s.ra; j <= jlast; ++j) {
        for (int g0 = 0; g0 <= jhi - R; g0 += 32) {
            // lane 0 takes the group's first column in kernel order
            const int c = ks.nearest ? R + g0 + lane : jhi - g0 - lane;
            bool contrib = false;
            uint32_t col = 0u;
            if ((ks.nearest ? c <= jhi : c >= R) &&
                YORO_BOUND(j >= 0 && j < s.slots && c >= 0 && c < s.wpad, kBadHoles)) {
                const int i = j * s.wpad + c;
                const bool reached = (s.bits[j * s.nwords + (c >> 5)] >> (c & 31)) & 1u;
                contrib = reached && !(__uint_as_float(s.zt[i]) < d_occ);  // not foreground (O2)
                if (contrib) col = s.rgba[i];
            }
            uint32_t cm = __ballot_sync(0xffffffffu, contrib);
            while (cm) {  // contributors in kernel order
                const int k = __ffs(cm) - 1;
                cm &= cm - 1u;
                const uint32_t cc = __shfl_sync(0xffffffffu, col, k);
                if (!done) {
                    if (!f.add(cc)) {  // weight reached exactly 0
                        res = f.result();
                        done = true;
                    } else {
                        uint32_t out;
                        if (f.wrem <= kSettleFrom && f.settled(out)) {
                            res = out;
                            done = true;
                        }
                    }
                }
                if (__all_sync(0xffffffffu, done)) return res;
            }
        }
    }
    if (!done) res = f.any() ? f.result() : (YORO_BOUND(R < s.wpad, kBadHoles) ? s.crow(v)[R] : 0u);
    return res;
}

// Hole fill of a one-pixel crack (v, x): reached pixels at x-1 and x+1, so L = x-1,
// R = x+1, w = 2 and t = 1/2.  The kernel is rows v-1, v, v+1 (v - halo .. v + halo)
// times columns min(x+3, W-1) .. x+1 (or x+1 .. x+3 nearest first); all slots are
// visited in the same order as fill_from_edges,
// without early exits.  A slot that does not contribute (outside the image, a hole, or
// nearer than the occluder) is given weight 0, which leaves acc and wrem unchanged
// exactly, so the result equals the general loop's.
template <bool VAR>
__device__ __forceinline__ uint32_t fill_crack(int x, int v, int h, int w, const Window& s,
                                               const KernelShape<VAR>& ks)
{
    const float d_occ = __uint_as_float(s.zrow(v)[x - 1]);
    FillAcc f;
    f.init(0.5f);
#pragma unroll
    for (int k = 0; k <= 2 * ks.halo; ++k) {
        const int vv = v - ks.halo + k;
        const bool row_in = vv >= 0 && vv < h;
        // a valid row to read when vv is outside
        const int vr = (row_in && YORO_BOUND(vv - s.ra >= 0 && vv - s.ra < s.slots, kBadHoles)) ? vv : v;
        const uint32_t* b = s.brow(vr);
        const uint32_t* zr = s.zrow(vr);
        const uint32_t* cr = s.crow(vr);
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const int col = ks.nearest ? x + 1 + c : x + 3 - c;
            const bool col_in = col < w;
            const int cc = col_in ? col : x + 1;
            const bool reached = (b[cc >> 5] >> (cc & 31)) & 1u;
            const bool contributes = row_in && col_in && reached && !(__uint_as_float(zr[cc]) < d_occ);
            f.add_if(contributes, cr[cc]);
        }
    }
    return f.any() ? f.result() : s.crow(v)[x + 1];
}

// Interior holes of 32-pixel word g of a band row with reached bitmask bv and last
// reached column `last`: one-pixel cracks (both neighbours reached) in cm, wider holes
// in gm.  Holes right of `last` are border holes and in neither.
__device__ __forceinline__ void hole_masks(const uint32_t* bv, int g, int nwords, int last, uint32_t& cm,
                                           uint32_t& gm)
{
    const uint32_t reach = bv[g];
    const uint32_t prev = g > 0 ? bv[g - 1] : 0u;
    const uint32_t next = g + 1 < nwords ? bv[g + 1] : 0u;
    const int rem = last - (g << 5);
    const uint32_t inb = rem >= 31 ? ~0u : (rem >= 0 ? ((2u << rem) - 1u) : 0u);
    const uint32_t hw = ~reach & inb;
    const uint32_t left = (reach << 1) | (prev >> 31);   // bit i: column 32g + i - 1 reached
    const uint32_t right = (reach >> 1) | (next << 31);  // bit i: column 32g + i + 1 reached
    cm = hw & left & right;
    gm = hw & ~cm;
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

// P1 (Alg. 1 closed form, Alg. 2 nearest kept) over the window's nr rows.
//
// Alg. 2 keeps, per target, the nearest source, on equal depth the one met first.  In
// one row that is the source with the largest column: with k = fx * ipd >= 0,
// Q = RN(k / zc) does not grow with the clamped depth zc, and the target
// floor(RN(x + 0.5 - Q)) rises by at least one per column at fixed Q (for targets in
// [0, 2^22) the rounding unit is at most 1/2, and a round-half-even tie resolves the
// same way one column apart).  So if sources x1 < x2 reach
// one target, Q1 < Q2, i.e. zc1 > zc2: the right one is strictly nearer, and equal
// depths never meet.  Each source therefore takes an atomic maximum of its column into
// its target's word (one native 32-bit shared atomic), and the depth is fetched for
// the winner alone in P2.
//
// Two forms deal the window's pixels to the threads.  In the two-column form each
// thread takes the columns x = tid and x + NT of every window row: consecutive lanes take
// consecutive columns, so a warp's loads of one row are one 128-byte line; a column's
// centre x + 0.5 and its depth pointer are set once, so a pixel costs only its row step;
// and the thread issues the loads of U = 5 rows of both columns before it processes any
// (a 15-row window is three groups; the rows left over form one group of their own
// height).  At 1832 columns it executes 12 % fewer
// instructions than the flat form below and keeps more loads in flight (measured
// against one column at a time with 3 to 15 rows per group, two columns with 3, 4 or 7
// rows, and (row group, column) units dealt round-robin).  But a thread's share is whole
// columns, so where the columns do not split evenly over the threads the flat form,
// pixels dealt round-robin in memory order, balances better.
template <int NT, int U>
__device__ __forceinline__ void scatter_rows(const FrameArgs& f, const float* dcol, int j, int nr, int x, float xc,
                                             bool two, int* srow, int wpad, uint32_t near_m1, uint32_t far_m1)
{
    const int w = f.w;
    float z[2][U];
#pragma unroll
    for (int c = 0; c < 2; ++c)
#pragma unroll
        for (int u = 0; u < U; ++u)
            z[c][u] = ((c == 0 || two) && YORO_BOUND(j + u < nr, kBadScatter))
                          ? __ldg(dcol + c * NT + (size_t)u * w)
                          : 0.0f;
#pragma unroll
    for (int c = 0; c < 2; ++c)
#pragma unroll
        for (int u = 0; u < U; ++u) {
            if (c == 0 || two) {
                uint32_t zb;
                const int xt = disparity_target(z[c][u], __fadd_rn(xc, (float)(c * NT)), f.k, near_m1, far_m1,
                                                f.half_m, zb);
                if ((unsigned)xt < (unsigned)w && YORO_BOUND(j + u < nr, kBadScatter))
                    atomicMax(srow + u * wpad + xt, x + c * NT);
            }
        }
}

// Next pixel of a flat (row, column) enumeration of a region `rw` columns wide dealt
// round-robin: advance by `dq` columns and `dr` rows (the stride split as rows and a
// remainder), carrying a row.
__device__ __forceinline__ void advance(int& r, int& q, int dr, int dq, int rw)
{
    q += dq;
    r += dr;
    if (q >= rw) {
        q -= rw;
        ++r;
    }
}

// The flat form over columns x0 .. w-1 of the window rows: pixel i = r * rw + q
// (rw = w - x0) goes to thread i mod NT, which issues the loads of U = 4 pixels before
// it processes any.
template <int NT, int U, bool FULL>
__device__ __forceinline__ void scatter_flat(const FrameArgs& f, const float* depth, int n, int i, int& r, int& q,
                                             int dr, int dq, int x0, int rw, int* src, int wpad, uint32_t near_m1,
                                             uint32_t far_m1)
{
    const int w = f.w;
    float z[U];
    int ru[U], xu[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
        ru[u] = r;
        xu[u] = x0 + q;
        z[u] = ((FULL || i + u * NT < n) && YORO_BOUND(i + u * NT < n, kBadScatter))
                   ? __ldg(depth + (size_t)r * w + x0 + q)
                   : 0.0f;
        advance(r, q, dr, dq, rw);
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
        if (FULL || i + u * NT < n) {
            uint32_t zb;
            const int xt = disparity_target(z[u], __fadd_rn((float)xu[u], 0.5f), f.k, near_m1, far_m1, f.half_m, zb);
            if ((unsigned)xt < (unsigned)w) atomicMax(src + ru[u] * wpad + xt, xu[u]);
        }
    }
}

template <int NT>
__device__ __forceinline__ void scatter_window(const FrameArgs& f, const float* depth, int nr, int* src, int wpad)
{
    constexpr int U = 5;
    const int w = f.w;
    const uint32_t near_m1 = __float_as_uint(f.near_) - 1u, far_m1 = __float_as_uint(f.far_) - 1u;
    // Columns of the two-column form: the first 2 NT of a frame at least that wide, else
    // all of them if no thread's share exceeds the mean share by more than a quarter
    // (2 NT / w or NT / w <= 5/4; at 1440 columns, 2 NT / w = 1.42 and the flat form
    // measured 3 % faster), else none.
    const int pc = w >= 2 * NT ? 2 * NT : (w > NT ? (5 * w >= 8 * NT ? w : 0) : (5 * w >= 4 * NT ? w : 0));
    const int x = threadIdx.x;
    if (x < pc) {
        const bool two = x + NT < pc;
        const float xc = __fadd_rn((float)x, 0.5f);  // exact: x < 2^23
        const float* dcol = depth + x;
        int* srow = src;
        int j = 0;
        for (; j + U <= nr; j += U) {  // every row of the group in the window
            scatter_rows<NT, U>(f, dcol, j, nr, x, xc, two, srow, wpad, near_m1, far_m1);
            dcol += (size_t)U * w;
            srow += U * wpad;
        }
        switch (nr - j) {  // the last rows as one group of their own height
        case 1: scatter_rows<NT, 1>(f, dcol, j, nr, x, xc, two, srow, wpad, near_m1, far_m1); break;
        case 2: scatter_rows<NT, 2>(f, dcol, j, nr, x, xc, two, srow, wpad, near_m1, far_m1); break;
        case 3: scatter_rows<NT, 3>(f, dcol, j, nr, x, xc, two, srow, wpad, near_m1, far_m1); break;
        case 4: scatter_rows<NT, 4>(f, dcol, j, nr, x, xc, two, srow, wpad, near_m1, far_m1); break;
        default: break;
        }
    }
    // the other columns (none at 1832 columns; 16 at 2064) in the flat form
    const int rw = w - pc;
    if (rw > 0) {
        constexpr int UF = 4;
        const int n = nr * rw;
        const int dr = NT / rw, dq = NT - dr * rw;
        int r = (int)threadIdx.x / rw, q = (int)threadIdx.x - r * rw;
        int i = threadIdx.x;
        for (; i + (UF - 1) * NT < n; i += UF * NT)  // every load of the group in range
            scatter_flat<NT, UF, true>(f, depth, n, i, r, q, dr, dq, pc, rw, src, wpad, near_m1, far_m1);
        if (i < n) scatter_flat<NT, UF, false>(f, depth, n, i, r, q, dr, dq, pc, rw, src, wpad, near_m1, far_m1);
    }
}

// P2 (resolve + gather) over the window: warp `warp` owns the 32-pixel words
// g = warp, warp + NW, ... of every row and takes RB rows per batch.  A reached target
// loads its source's depth (clamped as in P1) and color; ballots give the reached
// bitmasks.  Band rows send their reached pixels and hole mask to global memory right
// here; their holes are written in P3.  The loads of a batch are unconditional (a hole
// or a lane past the row end reads column 0, a batch row past the window reads the
// last window row), so the batch has no branches around its loads.
template <int RB, bool FULL, int NWI, int DX, bool ZT>
__device__ __forceinline__ void resolve_batch(const FrameArgs& f, const float* depth, const uint32_t* color,
                                              const Window& s, int g, int j0, int nb, int nr, int jb0, int jb1,
                                              uint32_t near_m1, uint32_t far_m1)
{
    // NWI words of the row batch at once: word g and, if NWI == 2, word g + DX / 32
    // (the next word the same warp owns), DX columns to the right.
    const int lane = threadIdx.x & 31;
    const int w = f.w, wpad = s.wpad;
    const int x = (g << 5) + lane;
    bool xin[NWI];
#pragma unroll
    for (int q = 0; q < NWI; ++q) xin[q] = x + q * DX < w;
    int sc[NWI][RB];
    float zs[NWI][RB];
    uint32_t cs[NWI][RB];
    // offsets advance by one row stride per row: no multiplies in the batch
    int so = j0 * wpad + x;  // shared-memory word of (row, x)
    int go = j0 * w;         // global pixel offset of the row in the window
#pragma unroll
    for (int u = 0; u < RB; ++u) {
#pragma unroll
        for (int q = 0; q < NWI; ++q)
            sc[q][u] = ((FULL || u < nb) && xin[q] && YORO_BOUND(so + q * DX < nr * wpad, kBadResolve))
                           ? (int)s.zt[so + q * DX]
                           : -1;
        so += wpad;
    }
#pragma unroll
    for (int u = 0; u < RB; ++u) {
#pragma unroll
        for (int q = 0; q < NWI; ++q) {
            const int o = go + max(sc[q][u], 0);
            zs[q][u] = 0.0f;
            cs[q][u] = 0u;
            if ((FULL || u < nb) && YORO_BOUND(o < nr * w, kBadResolve)) {
                zs[q][u] = __ldg(depth + o);
                cs[q][u] = __ldg(color + o);
            }
        }
        go += w;
    }
    so = j0 * wpad + x;
    int vo = (s.ra + j0) * w + x;  // frame pixel offset of (row, x)
#pragma unroll
    for (int u = 0; u < RB; ++u) {
        if (FULL || u < nb) {
            const int j = j0 + u;
            const bool band = j >= jb0 && j < jb1;
#pragma unroll
            for (int q = 0; q < NWI; ++q) {
                const bool reached = sc[q][u] >= 0;
                const uint32_t m = __ballot_sync(0xffffffffu, reached);
                const uint32_t zbits = clamped_depth_bits(zs[q][u], near_m1, far_m1);
                if (reached && YORO_BOUND(so + q * DX < nr * wpad, kBadResolve)) {
                    s.zt[so + q * DX] = zbits;
                    s.rgba[so + q * DX] = cs[q][u];
                }
                if (lane == 0 && YORO_BOUND(g + q * (DX >> 5) < s.nwords && j < nr, kBadResolve))
                    s.bits[j * s.nwords + g + q * (DX >> 5)] = m;
                // a band row: the pixel and its mask byte leave
                if (band && xin[q] && YORO_BOUND(vo + q * DX < f.h * w, kBadResolve)) {
                    if (reached) f.out[vo + q * DX] = cs[q][u];
                    f.mask[vo + q * DX] = reached ? 0 : 1;
                    if (ZT && f.zt_out) f.zt_out[vo + q * DX] = reached ? __uint_as_float(zbits) : 0.0f;
                }
            }
        }
        so += wpad;
        vo += w;
    }
}

// WIDE (windows wider than 2 NT words): the words from 2 NT on are dealt as (word, row
// batch) items over all warps instead of as a third word of the first warps (2064-wide
// frames: 29.0 -> 27.5 us per frame).  A separate instantiation, so that the code of the
// common width is untouched (compiled into one kernel the extra loop cost 1832-wide
// frames 2.5 %).
template <int NT, bool ZT, bool WIDE = false>
__device__ __forceinline__ void resolve_window(const FrameArgs& f, const float* depth, const uint32_t* color,
                                               int nr, int y0, int y1, const Window& s)
{
    constexpr int NW = NT / 32, RB = 3;  // 15-row windows: five full batches (2..8 measured)
    constexpr int DX = 32 * NW;          // columns between the two words a warp takes at once
    const int warp = threadIdx.x >> 5;
    const uint32_t near_m1 = __float_as_uint(f.near_) - 1u, far_m1 = __float_as_uint(f.far_) - 1u;
    const int jb0 = y0 - s.ra, jb1 = y1 - s.ra;  // band rows of the window: [jb0, jb1)
    for (int g = warp; g < (WIDE ? min(s.nwords, 2 * NW) : s.nwords); g += 2 * NW) {
        const bool two = g + NW < s.nwords;  // warp-uniform
        int j0 = 0;
        for (; j0 + RB <= nr; j0 += RB) {
            if (two) resolve_batch<RB, true, 2, DX, ZT>(f, depth, color, s, g, j0, RB, nr, jb0, jb1, near_m1, far_m1);
            else resolve_batch<RB, true, 1, DX, ZT>(f, depth, color, s, g, j0, RB, nr, jb0, jb1, near_m1, far_m1);
        }
        if (j0 < nr) {
            if (two) resolve_batch<RB, false, 2, DX, ZT>(f, depth, color, s, g, j0, nr - j0, nr, jb0, jb1, near_m1,
                                                     far_m1);
            else resolve_batch<RB, false, 1, DX, ZT>(f, depth, color, s, g, j0, nr - j0, nr, jb0, jb1, near_m1,
                                                     far_m1);
        }
    }
    if (WIDE) {
        const int nbat = (nr + RB - 1) / RB;
        for (int it = warp; it < (s.nwords - 2 * NW) * nbat; it += NW) {
            const int gw = 2 * NW + it / nbat, j0 = (it - (it / nbat) * nbat) * RB;
            if (j0 + RB <= nr)
                resolve_batch<RB, true, 1, DX, ZT>(f, depth, color, s, gw, j0, RB, nr, jb0, jb1, near_m1, far_m1);
            else
                resolve_batch<RB, false, 1, DX, ZT>(f, depth, color, s, gw, j0, nr - j0, nr, jb0, jb1, near_m1,
                                                    far_m1);
        }
    }
}

// One band [y0, y1) of one frame; shared memory holds the window rows ra..rb
// (ra = y0-1 or 0, rb = y1 or h-1).  Ends with a barrier, so the next band may reuse
// shared memory.
template <int NT, bool VAR>
__device__ __forceinline__ void fill_band(const FrameArgs& f, int y0, int y1, const Window& s, int* ctr,
                                          int* rowinfo);

template <int NT, bool VAR, bool ZT, bool WIDE = false>
__device__ __forceinline__ void run_band(const FrameArgs& f, int y0, int y1, Window s, int* ctr, int* rowinfo)
{
    constexpr int NW = NT / 32;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int w = f.w, h = f.h;
    const KernelShape<VAR> ks(f);
    const int ra = max(y0 - ks.halo, 0), rb = min(y1 - 1 + ks.halo, h - 1);
    const int nr = rb - ra + 1;
    s.ra = ra;
    const float* depth = f.depth + (size_t)ra * w;
    const uint32_t* color = f.color + (size_t)ra * w;

    if (f.bulk && lane == 0) {  // one depth row, then its color row, per warp
        for (int j = warp; j < nr; j += NW) {
            prefetch_l2(depth + (size_t)j * w, (uint32_t)w * 4u);
            prefetch_l2(color + (size_t)j * w, (uint32_t)w * 4u);
        }
    }
    {
        uint4* z4 = reinterpret_cast<uint4*>(s.zt);  // four words per 16 bytes; wpad % 8 == 0
        const int n4 = nr * (s.wpad >> 2);
        const uint4 e = make_uint4(~0u, ~0u, ~0u, ~0u);
        for (int i = tid; i < n4; i += NT) z4[i] = e;
        if (tid == 0) *ctr = 0;
    }
    __syncthreads();

    // ---- P1: disparity and nearest-wins scatter of rows ra..rb
    scatter_window<NT>(f, depth, nr, reinterpret_cast<int*>(s.zt), s.wpad);
    __syncthreads();

    // ---- P2: resolve, gather depths and colors, reached bitmasks; band rows' reached
    // pixels and hole mask leave
    resolve_window<NT, ZT, WIDE>(f, depth, color, nr, y0, y1, s);
    __syncthreads();

    fill_band<NT, VAR>(f, y0, y1, s, ctr, rowinfo);
}

// P3 of one band [y0, y1) whose window (s.ra set) holds the reached pixels' depths and
// colors and every window row's reached bitmask.  Writes the band rows' holes to
// f.out (reached pixels and masks are not touched).  Ends with a barrier.
template <int NT, bool VAR>
__device__ __forceinline__ void fill_band(const FrameArgs& f, int y0, int y1, const Window& s, int* ctr,
                                          int* rowinfo)
{
    constexpr int NW = NT / 32;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int w = f.w, h = f.h;
    const int nwords = s.nwords;
    const KernelShape<VAR> ks(f);

    // ---- P3a: per band row (one warp per row; rows with every pixel reached are done):
    // its last reached column, the border holes right of it, and per 32-pixel word the
    // number of interior cracks and wider holes with their prefix sums within the row.  Border holes have no
    // background edge (R = W) and take the fallback, the color of the last reached pixel
    // (zero if the row has none).  Counts are packed as cracks | wider << 16: a band
    // holds fewer than 2^16 pixels.
    const int nb = y1 - y0;
    int* lastr = rowinfo;           // last reached column of band row vj
    int* rowoff = lastr + s.slots;  // holes of the band rows before row vj
    for (int vj = warp; vj < nb; vj += NW) {
        uint32_t tot = 0u;
        const int v = y0 + vj;
        const uint32_t* bv = s.brow(v);
        int last = -1;
        bool full = true;  // every pixel of the row reached
        for (int gg = lane; gg < nwords; gg += 32) {
            const uint32_t b = bv[gg];
            if (b) last = (gg << 5) + 31 - __clz(b);
            const uint32_t inrow = (gg == nwords - 1 && (w & 31)) ? (1u << (w & 31)) - 1u : ~0u;
            full = full && b == inrow;
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) last = max(last, __shfl_xor_sync(0xffffffffu, last, o));
        if (!__all_sync(0xffffffffu, full)) {  // warp-uniform
            const uint32_t border = last >= 0 ? s.crow(v)[last] : 0u;
            uint32_t* orow = f.out + (size_t)v * w;
            for (int x = last + 1 + lane; x < w; x += 32) orow[x] = border;
            if (lane == 0) lastr[vj] = last;
            uint32_t* pre = s.pre + vj * nwords;
            for (int g0 = 0; g0 < nwords; g0 += 32) {
                const int g = g0 + lane;
                uint32_t c = 0u;
                if (g < nwords) {
                    uint32_t cm, gm;
                    hole_masks(bv, g, nwords, last, cm, gm);
                    c = (uint32_t)__popc(cm) | ((uint32_t)__popc(gm) << 16);
                }
                uint32_t sc = c;  // inclusive scan over the lanes
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const uint32_t y = __shfl_up_sync(0xffffffffu, sc, o);
                    if (lane >= o) sc += y;
                }
                if (g < nwords) pre[g] = tot + sc - c;
                tot += __shfl_sync(0xffffffffu, sc, 31);
            }
        }
        if (lane == 0) rowoff[vj] = (int)tot;
    }
    __syncthreads();
    if (warp == 0) {  // exclusive scan of the row totals; the band total goes to ctr[1]
        uint32_t run = 0u;
        for (int c0 = 0; c0 < nb; c0 += 32) {
            const uint32_t c = c0 + lane < nb ? (uint32_t)rowoff[c0 + lane] : 0u;
            uint32_t sc = c;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t y = __shfl_up_sync(0xffffffffu, sc, o);
                if (lane >= o) sc += y;
            }
            if (c0 + lane < nb) rowoff[c0 + lane] = (int)(run + sc - c);
            run += __shfl_sync(0xffffffffu, sc, 31);
        }
        if (lane == 0) ctr[1] = (int)run;
    }
    __syncthreads();

    // ---- P3b: fill of the interior holes (Alg. 3, Eq. 6).  The band's wider holes, then
    // its cracks, in row-major order, are dealt in chunks to whichever warp takes the next
    // chunk from a shared counter, so a wide disocclusion is spread over many warps and
    // every chunk but the last of each kind is full: 32 wider-hole pixels (one per lane),
    // or 64 cracks (two consecutive ones per lane: a crack's nine-slot fill is short, so
    // the search that locates it is a large part of its cost, and the second crack is
    // found from the first by the next crack bit of its row; 1832x1920, four streams:
    // 19.67 -> 19.52 us per frame, four per lane 20.52).  A lane finds its first hole by
    // binary search over the row and word prefix sums.
    {
        const uint32_t tot = (uint32_t)ctr[1];
        const int tc = (int)(tot & 0xffffu), tg = (int)(tot >> 16);
        const int ng = (tg + 31) >> 5, nchunks = ng + ((tc + 63) >> 6);
        // hole idx of the kind selected by sh (16: wider holes, 0: cracks) -> band row vj,
        // its rank r in the row, word g, rank k in the word, the word's hole masks
        auto locate = [&](int idx, int sh, int& vj, int& r, int& g, int& k, uint32_t& cm, uint32_t& gm) {
            // band row: the last row whose offset is <= idx
            int lo = 0, hi = nb - 1;
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if ((int)(((uint32_t)rowoff[mid] >> sh) & 0xffffu) <= idx) lo = mid;
                else hi = mid - 1;
            }
            vj = lo;
            r = idx - (int)(((uint32_t)rowoff[vj] >> sh) & 0xffffu);
            // word of the row: the last word whose prefix is <= r
            const uint32_t* pre = s.pre + vj * nwords;
            lo = 0;
            hi = nwords - 1;
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if ((int)((pre[mid] >> sh) & 0xffffu) <= r) lo = mid;
                else hi = mid - 1;
            }
            g = lo;
            k = r - (int)((pre[g] >> sh) & 0xffffu);
            hole_masks(s.brow(y0 + vj), g, nwords, lastr[vj], cm, gm);
        };
        for (;;) {
            int chunk = 0;
            if (lane == 0) chunk = atomicAdd(ctr, 1);
            chunk = __shfl_sync(0xffffffffu, chunk, 0);
            if (chunk >= nchunks) break;
            if (chunk < ng) {  // 32 pixels of wider holes, one per lane (warp-uniform branch)
                const int idx = (chunk << 5) + lane;
                bool act = idx < tg;  // lane 0 is always active
                int v = 0, x = 0;
                if (act) {
                    int vj, r, g, k;
                    uint32_t cm, gm;
                    locate(idx, 16, vj, r, g, k, cm, gm);
                    v = y0 + vj;
                    x = (g << 5) + nth_set_bit(gm, k);
                    // the located pixel is a hole of the band row (checked in the debug-bounds build)
                    act = YORO_BOUND((unsigned)x < (unsigned)w && !((s.brow(v)[x >> 5] >> (x & 31)) & 1u),
                                     kBadHoles);
                }
                uint32_t o = 0u;
                int L = -1, R = 0;
                if (act) find_edges(x, v, s, w, L, R);
                // one hole for the whole chunk: its kernel is scanned once by the warp
                const int v0 = __shfl_sync(0xffffffffu, v, 0), L0 = __shfl_sync(0xffffffffu, L, 0),
                          R0 = __shfl_sync(0xffffffffu, R, 0);
                if (__all_sync(0xffffffffu, !act || (v == v0 && L == L0 && R == R0)))
                    o = fill_hole_warp<VAR>(x, act, v0, L0, R0, h, w, s, ks);
                else if (act)
                    o = fill_from_edges<VAR>(x, v, L, R, h, w, s, ks);
                if (act && YORO_BOUND(v >= y0 && v < y1, kBadHoles)) f.out[(size_t)v * w + x] = o;
            } else {  // 64 cracks, two consecutive ones per lane
                const int idx = ((chunk - ng) << 6) + 2 * lane;
                bool act0 = idx < tc, act1 = idx + 1 < tc;
                int v0 = 0, x0 = 0, v1 = 0, x1 = 0;
                if (act0) {
                    int vj, r, g, k;
                    uint32_t cm, gm;
                    locate(idx, 0, vj, r, g, k, cm, gm);
                    const int b0 = nth_set_bit(cm, k);
                    v0 = y0 + vj;
                    x0 = (g << 5) + b0;
                    act0 = YORO_BOUND((unsigned)x0 < (unsigned)w && !((s.brow(v0)[x0 >> 5] >> (x0 & 31)) & 1u),
                                      kBadHoles);
                    if (act1) {
                        const int rowc = (vj + 1 < nb ? (int)((uint32_t)rowoff[vj + 1] & 0xffffu) : tc) -
                                         (int)((uint32_t)rowoff[vj] & 0xffffu);  // cracks of row vj
                        if (r + 1 < rowc) {  // the next crack of the same row: the next crack bit
                            const uint32_t* bv = s.brow(v0);
                            uint32_t rest = b0 == 31 ? 0u : (cm & (~0u << (b0 + 1)));
                            int g1 = g;
                            while (!rest && YORO_BOUND(g1 + 1 < nwords, kBadHoles)) {
                                ++g1;
                                hole_masks(bv, g1, nwords, lastr[vj], rest, gm);
                            }
                            v1 = v0;
                            x1 = (g1 << 5) + __ffs(rest) - 1;
                        } else {  // the first crack of a later row
                            locate(idx + 1, 0, vj, r, g, k, cm, gm);
                            v1 = y0 + vj;
                            x1 = (g << 5) + nth_set_bit(cm, k);
                        }
                        act1 = YORO_BOUND(
                            (unsigned)x1 < (unsigned)w && !((s.brow(v1)[x1 >> 5] >> (x1 & 31)) & 1u), kBadHoles);
                    }
                }
                if (act0 && YORO_BOUND(v0 >= y0 && v0 < y1, kBadHoles))
                    f.out[(size_t)v0 * w + x0] = fill_crack<VAR>(x0, v0, h, w, s, ks);
                if (act1 && YORO_BOUND(v1 >= y0 && v1 < y1, kBadHoles))
                    f.out[(size_t)v1 * w + x1] = fill_crack<VAR>(x1, v1, h, w, s, ks);
            }
        }
    }
    __syncthreads();
}

// Shared-memory layout of a window of `slots` rows (see fused_smem_bytes).
__device__ __forceinline__ Window window_layout(unsigned char* smem, int slots, int wpad, int w, int*& ctr,
                                                int*& rowinfo)
{
    Window s;
    s.zt = reinterpret_cast<uint32_t*>(smem);
    s.rgba = s.zt + slots * wpad;
    s.bits = s.rgba + slots * wpad;
    s.wpad = wpad;
    s.nwords = (w + 31) >> 5;
    s.ra = 0;
    s.slots = slots;
    s.pre = s.bits + slots * ((wpad + 31) / 32);
    ctr = reinterpret_cast<int*>(s.pre + slots * ((wpad + 31) / 32));
    rowinfo = ctr + 4;
    return s;
}

template <int NT, int MINB, bool VAR, bool ZT = false, bool WIDE = false>
__global__ void __launch_bounds__(NT, MINB) fused_single(FrameArgs f, int wpad)
{
    extern __shared__ __align__(128) unsigned char smem_raw[];
    int *ctr, *rowinfo;
    const Window s = window_layout(smem_raw, f.band + 2 * KernelShape<VAR>(f).halo, wpad, f.w, ctr, rowinfo);
    const int nbands = (f.h + f.band - 1) / f.band;
    for (int b = blockIdx.x; b < nbands; b += gridDim.x) {
        const int y0 = b * f.band;
        run_band<NT, VAR, ZT, WIDE>(f, y0, min(y0 + f.band, f.h), s, ctr, rowinfo);
    }
}

template <int NT, int MINB, bool ZT = false, bool WIDE = false>
__global__ void __launch_bounds__(NT, MINB) fused_batch(const __grid_constant__ BatchArgs a, int wpad)
{
    extern __shared__ __align__(128) unsigned char smem_raw[];
    for (int item = blockIdx.x; item < a.total_items; item += gridDim.x) {
        int lo = 0, hi = a.n - 1;  // frame whose item range holds `item`
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (a.item_start[mid] <= item) lo = mid;
            else hi = mid - 1;
        }
        const FrameArgs& f = a.f[lo];
        int *ctr, *rowinfo;
        // the frame's own row stride: a narrower frame fits more rows (f.band) in the
        // shared memory sized for max_band rows of the widest
        const Window s = window_layout(smem_raw, f.band + 2, (f.w + 7) / 8 * 8, f.w, ctr, rowinfo);
        const int y0 = (item - a.item_start[lo]) * f.band;
        run_band<NT, false, ZT, WIDE>(f, y0, min(y0 + f.band, f.h), s, ctr, rowinfo);
    }
}

// P3 alone over an image that is already resolved in global memory: the reached pixels'
// colors in f.out, their depths in zt, the hole mask in f.mask (the row-downsampled
// intermediate buffer's and the general pose's full-resolution image).  Each band's window
// is loaded (the reached bitmasks by ballot over the mask bytes, depths and colors of the
// reached pixels; each warp takes four 32-pixel words at a time, their loads issued
// before any is used), then filled exactly as the fused kernel fills its bands.  VAR as
// in the fused kernel: false compiles the paper's kernel shape as constants.
template <int NT, bool VAR>
__global__ void __launch_bounds__(NT, 1) fill_only(FrameArgs f, const float* __restrict__ zt, int wpad)
{
    extern __shared__ __align__(128) unsigned char smem_raw[];
    constexpr int NW = NT / 32;
    int *ctr, *rowinfo;
    const KernelShape<VAR> ks(f);
    Window s = window_layout(smem_raw, f.band + 2 * ks.halo, wpad, f.w, ctr, rowinfo);
    const int w = f.w, h = f.h, nwords = s.nwords;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nbands = (h + f.band - 1) / f.band;
    for (int b = blockIdx.x; b < nbands; b += gridDim.x) {
        const int y0 = b * f.band, y1 = min(y0 + f.band, h);
        const int ra = max(y0 - ks.halo, 0), rb = min(y1 - 1 + ks.halo, h - 1);
        const int nr = rb - ra + 1;
        s.ra = ra;
        const int items = nr * nwords;
        for (int it0 = warp; it0 < items; it0 += 4 * NW) {
            uint32_t mk[4], zv[4], cv[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int it = it0 + q * NW;
                const int j = it / nwords, g = it - j * nwords;
                const int x = (g << 5) + lane;
                const size_t o = (size_t)(ra + j) * w + x;
                const bool ld = it < items && x < w;
                mk[q] = ld ? f.mask[o] : 1u;
                zv[q] = ld ? __float_as_uint(zt[o]) : 0u;
                cv[q] = ld ? f.out[o] : 0u;
            }
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int it = it0 + q * NW;
                if (it >= items) break;  // warp-uniform
                const int j = it / nwords, g = it - j * nwords;
                const int x = (g << 5) + lane;
                const bool reached = mk[q] == 0u;
                const uint32_t m = __ballot_sync(0xffffffffu, reached);
                if (lane == 0 && YORO_BOUND(j < s.slots, kBadHoles)) s.bits[j * nwords + g] = m;
                if (reached && YORO_BOUND(j * wpad + x < s.slots * wpad, kBadHoles)) {
                    s.zt[j * wpad + x] = zv[q];
                    s.rgba[j * wpad + x] = cv[q];
                }
            }
        }
        if (threadIdx.x == 0) *ctr = 0;
        __syncthreads();
        fill_band<NT, VAR>(f, y0, y1, s, ctr, rowinfo);
    }
}

// The band fill straight from a frame-wide z-buffer of 64-bit keys (clamped depth bits
// above the source pixel's index, the empty key at holes: the general pose's Alg. 2 over
// the frame): each band's window is loaded from the keys (reached bitmask, the depth from
// the key, the winner's color gathered from f.color), the band rows' colors of reached
// pixels and their hole mask leave for global memory, and the holes are filled as in
// fill_only.  It stands in for a gather pass that writes the image out and fill_only's
// reading it back.
template <int NT, bool VAR>
__global__ void __launch_bounds__(NT, 1) fill_keys(FrameArgs f, const unsigned long long* __restrict__ keys, int wpad)
{
    extern __shared__ __align__(128) unsigned char smem_raw[];
    constexpr int NW = NT / 32;
    int *ctr, *rowinfo;
    const KernelShape<VAR> ks(f);
    Window s = window_layout(smem_raw, f.band + 2 * ks.halo, wpad, f.w, ctr, rowinfo);
    const int w = f.w, h = f.h, nwords = s.nwords;
    const size_t n = (size_t)w * (size_t)h;  // source indices are below n (checked in the debug-bounds build)
    (void)n;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nbands = (h + f.band - 1) / f.band;
    for (int b = blockIdx.x; b < nbands; b += gridDim.x) {
        const int y0 = b * f.band, y1 = min(y0 + f.band, h);
        const int ra = max(y0 - ks.halo, 0), rb = min(y1 - 1 + ks.halo, h - 1);
        const int nr = rb - ra + 1;
        s.ra = ra;
        const int items = nr * nwords;
        for (int it0 = warp; it0 < items; it0 += 4 * NW) {
            unsigned long long kv[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int it = it0 + q * NW;
                const int j = it / nwords, g = it - j * nwords;
                const int x = (g << 5) + lane;
                kv[q] = (it < items && x < w) ? keys[(size_t)(ra + j) * w + x] : kEmptyKey;
            }
            uint32_t cv[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const uint32_t src = (uint32_t)kv[q];
                cv[q] = (kv[q] != kEmptyKey && YORO_BOUND(src < n, kBadPose)) ? __ldg(f.color + src) : 0u;
            }
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int it = it0 + q * NW;
                if (it >= items) break;  // warp-uniform
                const int j = it / nwords, g = it - j * nwords;
                const int x = (g << 5) + lane;
                const bool reached = kv[q] != kEmptyKey;
                const uint32_t m = __ballot_sync(0xffffffffu, reached);
                if (lane == 0 && YORO_BOUND(j < s.slots, kBadHoles)) s.bits[j * nwords + g] = m;
                if (reached && YORO_BOUND(j * wpad + x < s.slots * wpad, kBadHoles)) {
                    s.zt[j * wpad + x] = (uint32_t)(kv[q] >> 32);
                    s.rgba[j * wpad + x] = cv[q];
                }
                const int v = ra + j;
                if (v >= y0 && v < y1 && x < w) {  // a band row: the pixel and its mask byte leave
                    const size_t o = (size_t)v * w + x;
                    if (reached) f.out[o] = cv[q];
                    f.mask[o] = reached ? 0 : 1;
                }
            }
        }
        if (threadIdx.x == 0) *ctr = 0;
        __syncthreads();
        fill_band<NT, VAR>(f, y0, y1, s, ctr, rowinfo);
    }
}

// The row-downsampled intermediate buffer in one kernel: per band, the window rows'
// cells are reprojected into 64-bit cell keys in shared memory (after the window),
// every window pixel is sampled from its cell's winner into the window (depth, color,
// reached bitmask; the band rows' reached pixels and masks leave for global memory),
// and the band's holes are filled as the fused kernel fills them.  The steps and their
// rounding are those of imbuffer.cu's separate kernels (the reading is stated there).
template <int NT>
__global__ void __launch_bounds__(NT, 1) imb_band(FrameArgs f, int div, int interp, int wpad, int cells_off)
{
    extern __shared__ __align__(128) unsigned char smem_raw[];
    constexpr int NW = NT / 32;
    int *ctr, *rowinfo;
    const KernelShape<true> ks(f);
    const int slots = f.band + 2 * ks.halo;
    Window s = window_layout(smem_raw, slots, wpad, f.w, ctr, rowinfo);
    const int w = f.w, h = f.h, nwords = s.nwords, ws = (w + div - 1) / div;
    unsigned long long* cells = reinterpret_cast<unsigned long long*>(smem_raw + cells_off);  // after the window
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint32_t near_m1 = __float_as_uint(f.near_) - 1u, far_m1 = __float_as_uint(f.far_) - 1u;
    const float inv_s = 1.0f / (float)div;
    const int lg = __ffs(div) - 1;  // div is a power of two
    const int nbands = (h + f.band - 1) / f.band;
    for (int b = blockIdx.x; b < nbands; b += gridDim.x) {
        const int y0 = b * f.band, y1 = min(y0 + f.band, h);
        const int ra = max(y0 - ks.halo, 0), rb = min(y1 - 1 + ks.halo, h - 1);
        const int nr = rb - ra + 1;
        s.ra = ra;
        if (f.bulk && lane == 0) {  // one depth row, then its color row, per warp
            for (int j = warp; j < nr; j += NW) {
                prefetch_l2(f.depth + (size_t)(ra + j) * w, (uint32_t)w * 4u);
                prefetch_l2(f.color + (size_t)(ra + j) * w, (uint32_t)w * 4u);
            }
        }
        for (int i = threadIdx.x; i < nr * ws; i += NT) cells[i] = kEmptyKey;
        if (threadIdx.x == 0) *ctr = 0;
        __syncthreads();
        // cells: Alg. 1 on each cell's pixel, Alg. 2 by a 64-bit minimum of the key;
        // (row j, cell i) of flat index c advance without a division per cell
        const int dj = NT / ws, di = NT - dj * ws;
        int cj = (int)threadIdx.x / ws, ci = (int)threadIdx.x - cj * ws;
        for (int c = threadIdx.x; c < nr * ws; c += NT) {
            const int j = cj, i = ci;
            cj += dj;
            ci += di;
            if (ci >= ws) {
                ci -= ws;
                ++cj;
            }
            const int p = min(div * i + (div >> 1), w - 1);
            const uint32_t zb = clamped_depth_bits(__ldg(f.depth + (size_t)(ra + j) * w + p), near_m1, far_m1);
            const float disp = __fdiv_rn(f.k, __uint_as_float(zb));
            const float t = __fsub_rn(__fadd_rn((float)p, 0.5f), disp);
            const float tc = floorf(__fmul_rn(t, inv_s));
            if (tc >= 0.0f && tc < (float)ws && YORO_BOUND(c < slots * ws, kBadScatter))
                atomicMin(&cells[j * ws + (int)tc], zkey(zb, i));
        }
        __syncthreads();
        if (interp) {  // the winner's shift once per cell: its key's low word becomes disp
            for (int c = threadIdx.x; c < nr * ws; c += NT) {
                const unsigned long long key = cells[c];
                if (key != kEmptyKey) {
                    const uint32_t zb = (uint32_t)(key >> 32);
                    cells[c] = ((unsigned long long)zb << 32) | __float_as_uint(__fdiv_rn(f.k, __uint_as_float(zb)));
                }
            }
            __syncthreads();
        }
        // sampling: each window pixel from its cell's winner; warp per 32-pixel word
        for (int it = warp; it < nr * nwords; it += NW) {
            const int j = it / nwords, g = it - j * nwords;
            const int x = (g << 5) + lane;
            const int y = ra + j;
            const unsigned long long* krow = cells + j * ws;
            const uint32_t* crow = f.color + (size_t)y * w;
            unsigned long long key = kEmptyKey;
            if (x < w) key = krow[x >> lg];
            const bool reached = key != kEmptyKey;
            const uint32_t m = __ballot_sync(0xffffffffu, reached);
            if (lane == 0 && YORO_BOUND(j < slots, kBadResolve)) s.bits[j * nwords + g] = m;
            const bool band = y >= y0 && y < y1;
            if (band && x < w) f.mask[(size_t)y * w + x] = reached ? 0 : 1;
            if (!reached) continue;
            const uint32_t zb = (uint32_t)(key >> 32);
            const int cj = x >> lg;
            uint32_t col;
            if (!interp) {
                col = __ldg(crow + min(div * (int)(uint32_t)key + (x - div * cj), w - 1));
            } else {
                const float dj = __uint_as_float((uint32_t)key);  // disp of the winner
                const float off =
                    __fsub_rn(__fadd_rn((float)x, 0.5f), __fadd_rn((float)(div * cj), 0.5f * (float)div));
                const int nb = off < 0.0f ? cj - 1 : cj + 1;
                float d = dj;
                if (off != 0.0f && nb >= 0 && nb < ws && krow[nb] != kEmptyKey) {
                    const float dn = __uint_as_float((uint32_t)krow[nb]);
                    d = __fadd_rn(dj, __fmul_rn(__fsub_rn(dn, dj), __fmul_rn(fabsf(off), inv_s)));
                }
                const float u = __fadd_rn((float)x, d);
                if (u <= 0.0f) {
                    col = __ldg(crow);
                } else if (u >= (float)(w - 1)) {
                    col = __ldg(crow + w - 1);
                } else {
                    const float fl = floorf(u);
                    const int i0 = (int)fl;
                    const float fr = __fsub_rn(u, fl);
                    const uint32_t c0 = __ldg(crow + i0), c1 = __ldg(crow + i0 + 1);
                    col = 0u;
#pragma unroll
                    for (int ch = 0; ch < 4; ++ch) {
                        const float v0 = (float)((c0 >> (8 * ch)) & 255u), v1 = (float)((c1 >> (8 * ch)) & 255u);
                        col |= (uint32_t)rintf(__fadd_rn(v0, __fmul_rn(__fsub_rn(v1, v0), fr))) << (8 * ch);
                    }
                }
            }
            if (YORO_BOUND(j * wpad + x < slots * wpad, kBadResolve)) {
                s.zt[j * wpad + x] = zb;
                s.rgba[j * wpad + x] = col;
            }
            if (band) f.out[(size_t)y * w + x] = col;
        }
        __syncthreads();
        fill_band<NT, true>(f, y0, y1, s, ctr, rowinfo);
    }
}

// Two shapes: 1024 threads with one CTA per SM (large bands), or 512 threads with
// two CTAs per SM (bands small enough that two fit in shared memory).
constexpr int kBig = 1024;
constexpr int kSmall = 512;

}  // namespace

int fused_wpad(int w) { return ((w + 7) / 8) * 8; }

unsigned fused_status_take()
{
#ifdef YORO_DEBUG_BOUNDS
    unsigned v = 0, z = 0;
    if (cudaMemcpyFromSymbol(&v, g_status, sizeof v) != cudaSuccess ||
        cudaMemcpyToSymbol(g_status, &z, sizeof z) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return v;
#else
    return 0;
#endif
}

cudaError_t debug_selftest_launch(cudaStream_t stream)
{
    selftest_kernel<<<1, 32, 0, stream>>>();
    return cudaGetLastError();
}

bool debug_bounds_built()
{
#ifdef YORO_DEBUG_BOUNDS
    return true;
#else
    return false;
#endif
}

size_t fused_smem_bytes(int wpad, int band, int halo)
{
    const size_t slots = (size_t)band + 2 * (size_t)halo;
    // per pixel a source/depth word and a color word; per 32-pixel word a reached
    // bitmask and a hole prefix sum; two counters (16 bytes); per window row a last
    // reached column and a hole offset
    return slots * (size_t)wpad * 8 + slots * (size_t)((wpad + 31) / 32) * 8 + 16 + slots * 8;
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
    while (fused_smem_bytes(fused_wpad(wmax + 32), 1, 1) <= (size_t)smem_optin && wmax + 32 <= 65535) wmax += 32;
    lim->max_width = wmax;
    const void* fns[] = {(const void*)fused_single<kBig, 1, false>, (const void*)fused_single<kSmall, 2, false>,
                         (const void*)fused_single<kBig, 1, true>,  (const void*)fused_single<kSmall, 2, true>,
                         (const void*)fused_single<kBig, 1, false, true>, (const void*)fused_single<kSmall, 2, false, true>,
                         (const void*)fused_batch<kBig, 1>,         (const void*)fused_batch<kSmall, 2>,
                         (const void*)fused_batch<kBig, 1, true>,   (const void*)fused_batch<kSmall, 2, true>,
                         (const void*)fused_single<kBig, 1, false, false, true>,
                         (const void*)fused_batch<kBig, 1, false, true>,
                         (const void*)fill_only<kBig, false>,       (const void*)fill_only<kBig, true>,
                         (const void*)fill_keys<kBig, false>,       (const void*)fill_keys<kBig, true>,
                         (const void*)imb_band<kBig>};
    for (const void* fn : fns) {
        e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_optin);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

// Largest band whose rows fit the per-CTA shared memory.
static int max_band(const FusedLimits& lim, int wpad, int halo)
{
    if (wpad <= 0) return 1;
    int b = 1;
    while (b < 4096 && fused_smem_bytes(wpad, b + 1, halo) <= (size_t)lim.smem_per_block) ++b;
    return b;
}

// Band height for a w x h frame: enough bands for every SM, each as tall as shared
// memory allows up to that.  Two CTAs per SM when two such bands fit on an SM.
FusedShape fused_shape(const FusedLimits& lim, int w, int h, int halo)
{
    const int wpad = fused_wpad(w);
    const int bmax = max_band(lim, wpad, halo);
    FusedShape s;
    int band = (h + lim.sms - 1) / lim.sms;
    if (band > bmax) band = bmax;
    if (band < 1) band = 1;
    // two CTAs of half the band height, if they fit beside each other
    const int half = (band + 1) / 2;
    if (band >= 2 && 2 * (fused_smem_bytes(wpad, half, halo) + 1024) <= (size_t)lim.smem_per_sm) {
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
    const size_t smem = fused_smem_bytes(wpad, f.band, f.halo);
    const bool var = f.halo != 1 || f.nearest != 0;  // a Patcher variant: its own instantiation
    const int nbands = (f.h + f.band - 1) / f.band;
    const int slots = lim.sms * (two_per_sm ? 2 : 1);
    const int grid = nbands < slots ? nbands : slots;
    if (f.zt_out && var) return cudaErrorInvalidValue;  // the depth output exists for the default kernel
    if (two_per_sm) {
        if (f.zt_out) fused_single<kSmall, 2, false, true><<<grid, kSmall, smem, stream>>>(f, wpad);
        else if (var) fused_single<kSmall, 2, true><<<grid, kSmall, smem, stream>>>(f, wpad);
        else fused_single<kSmall, 2, false><<<grid, kSmall, smem, stream>>>(f, wpad);
    } else {
        if (f.zt_out) fused_single<kBig, 1, false, true><<<grid, kBig, smem, stream>>>(f, wpad);
        else if (var) fused_single<kBig, 1, true><<<grid, kBig, smem, stream>>>(f, wpad);
        else if ((f.w + 31) / 32 > 2 * (kBig / 32))  // wider than 2 words per warp
            fused_single<kBig, 1, false, false, true><<<grid, kBig, smem, stream>>>(f, wpad);
        else fused_single<kBig, 1, false><<<grid, kBig, smem, stream>>>(f, wpad);
    }
    return cudaGetLastError();
}

cudaError_t fused_launch_batch(const BatchArgs& a, int wmax, const FusedLimits& lim, cudaStream_t stream, bool zt)
{
    const int wpad = fused_wpad(wmax);
    const size_t smem = fused_smem_bytes(wpad, a.max_band, 1);  // batch frames use the default kernel
    const bool two = 2 * (smem + 1024) <= (size_t)lim.smem_per_sm;
    // One CTA per (frame, band) item: the hardware block scheduler hands the next item to
    // whichever SM frees up first, so bands with heavy disocclusions do not hold back the
    // rest of the batch.
    const int grid = a.total_items;
    if (grid < 1) return cudaSuccess;
    if (two) {
        if (zt) fused_batch<kSmall, 2, true><<<grid, kSmall, smem, stream>>>(a, wpad);
        else fused_batch<kSmall, 2><<<grid, kSmall, smem, stream>>>(a, wpad);
    } else {
        if (zt) fused_batch<kBig, 1, true><<<grid, kBig, smem, stream>>>(a, wpad);
        else if ((wmax + 31) / 32 > 2 * (kBig / 32))  // a frame wider than 2 words per warp
            fused_batch<kBig, 1, false, true><<<grid, kBig, smem, stream>>>(a, wpad);
        else fused_batch<kBig, 1><<<grid, kBig, smem, stream>>>(a, wpad);
    }
    return cudaGetLastError();
}

int fused_max_band(const FusedLimits& lim, int w, int halo) { return max_band(lim, fused_wpad(w), halo); }

static size_t imb_cells_offset(int w, int band, int halo)
{
    return (fused_smem_bytes(fused_wpad(w), band, halo) + 15) & ~(size_t)15;
}

size_t imb_band_smem_bytes(int w, int band, int halo, int div)
{
    const int ws = (w + div - 1) / div;
    return imb_cells_offset(w, band, halo) + (size_t)(band + 2 * halo) * (size_t)ws * sizeof(unsigned long long);
}

int imb_band_max(const FusedLimits& lim, int w, int halo, int div)
{
    int b = 0;
    while (b < 4096 && imb_band_smem_bytes(w, b + 1, halo, div) <= (size_t)lim.smem_per_block) ++b;
    return b;
}

cudaError_t imb_band_launch(FrameArgs f, int div, int interp, const FusedLimits& lim, cudaStream_t stream)
{
    const int per_sm = (f.h + lim.sms - 1) / lim.sms;
    f.band = max(1, min(imb_band_max(lim, f.w, f.halo, div), per_sm));
    const size_t smem = imb_band_smem_bytes(f.w, f.band, f.halo, div);
    const int nbands = (f.h + f.band - 1) / f.band;
    const int grid = nbands < lim.sms ? nbands : lim.sms;
    if (grid < 1) return cudaSuccess;
    imb_band<kBig><<<grid, kBig, smem, stream>>>(f, div, interp, fused_wpad(f.w),
                                                 (int)imb_cells_offset(f.w, f.band, f.halo));
    return cudaGetLastError();
}

cudaError_t fill_only_launch(FrameArgs f, const float* zt, const FusedLimits& lim, cudaStream_t stream)
{
    const int wpad = fused_wpad(f.w);
    // bands as tall as shared memory allows, but at least one per SM
    const int per_sm = (f.h + lim.sms - 1) / lim.sms;
    f.band = max(1, min(max_band(lim, wpad, f.halo), per_sm));
    const size_t smem = fused_smem_bytes(wpad, f.band, f.halo);
    const int nbands = (f.h + f.band - 1) / f.band;
    const int grid = nbands < lim.sms ? nbands : lim.sms;
    if (grid < 1) return cudaSuccess;
    if (f.halo == 1 && !f.nearest) fill_only<kBig, false><<<grid, kBig, smem, stream>>>(f, zt, wpad);
    else fill_only<kBig, true><<<grid, kBig, smem, stream>>>(f, zt, wpad);
    return cudaGetLastError();
}

cudaError_t fill_keys_launch(FrameArgs f, const unsigned long long* keys, const FusedLimits& lim, cudaStream_t stream)
{
    const int wpad = fused_wpad(f.w);
    // bands as tall as shared memory allows, but at least one per SM
    const int per_sm = (f.h + lim.sms - 1) / lim.sms;
    f.band = max(1, min(max_band(lim, wpad, f.halo), per_sm));
    const size_t smem = fused_smem_bytes(wpad, f.band, f.halo);
    const int nbands = (f.h + f.band - 1) / f.band;
    const int grid = nbands < lim.sms ? nbands : lim.sms;
    if (grid < 1) return cudaSuccess;
    if (f.halo == 1 && !f.nearest) fill_keys<kBig, false><<<grid, kBig, smem, stream>>>(f, keys, wpad);
    else fill_keys<kBig, true><<<grid, kBig, smem, stream>>>(f, keys, wpad);
    return cudaGetLastError();
}

}  // namespace yoro
