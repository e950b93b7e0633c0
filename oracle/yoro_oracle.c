/*
 * CPU oracle for second-eye synthesis (YORO, "You Only Render Once").
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the CPU
 * baseline of the benchmark load this file.  The CUDA library never includes,
 * links or calls it, and it shares no header, helper or constant table with it.
 *
 * Plain, slow and sequential on purpose: every step is the paper's definition
 * written out in the order the paper gives, so it can be checked against the
 * paper by eye.  The row loops of the base path carry OpenMP pragmas: the default
 * build ignores them (one thread); the all-core CPU baseline compiles the same file
 * with -fopenmp, which only splits independent rows over threads (each row writes
 * its own outputs and reads earlier steps' arrays), so its results are the same.  Compiled with -O2 -ffp-contract=off and no fast-math, so every
 * float operation below is one IEEE binary32 operation rounded to nearest even.
 *
 * Precision: binary32 throughout.  The method turns floating point into integers
 * (a target column, a winning source, an 8-bit color), and those decisions are
 * taken in the precision of the CUDA path so that both sides agree exactly.
 *
 * Frame convention: the source is the LEFT eye and the output is the RIGHT eye.
 * The paper's examples use the right eye as source (pixels move +x, background at
 * -x); here pixels move -x and the background side of a hole is +x, so every
 * left/right choice of the paper is mirrored.
 *
 * Pins (tests that tie this file to the paper and to mathematics, not to itself):
 *   oracle_disparity     IPD = 0 identity; fronto-parallel plane closed-form shift;
 *                        analytic ray-cast of the right eye on tiny scenes.
 *   oracle_forward_warp  brute-force argmin over co-mapped sources (nearer wins,
 *                        lower source column on equal depth); ray-cast visibility.
 *   oracle_resolve       IPD = 0 identity; plane closed form.
 *   oracle_hole_edges    brute force nearest valid column on each side.
 *   oracle_fill          closed forms: one contributing candidate returns its color;
 *                        two contributors blend as c2 + (c1 - c2) / (1.5 - 0.3 t);
 *                        the geometric closed form sum q^i c_i / sum q^i (exact
 *                        rationals) for every kernel height and column order;
 *                        depth gate, kernel extent, row order and the fallback are
 *                        checked by hand-built cases.  Beyond those small cases the
 *                        fill on general inputs is parity unpinned: it follows the
 *                        literal reading of Algorithm 3 and Eq. 6 stated below.
 */
#include <math.h>
#include <stddef.h>
#ifdef _OPENMP
#include <omp.h>
#endif
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* Threads the row loops run on: 1 in the default build, the OpenMP team size in the
 * all-core build. */
int oracle_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/*
 * Algorithm 1 (Reprojector stage 1) in closed form, per source pixel (y, x).
 *
 * Eq. 5 maps a source pixel to the other eye with M = (VP_left)^-1 VP_right.  For
 * two pinhole eyes with the same intrinsics, parallel axes and a baseline of ipd
 * along +x, back-projecting pixel centre x + 0.5 at depth z gives
 * X = (x + 0.5 - cx) z / fx, and projecting into the eye at +ipd gives
 * x_R + 0.5 = fx (X - ipd) / z + cx = (x + 0.5) - fx ipd / z, with y and z
 * unchanged (observation O1: motion is along x only, in one direction).
 *
 *   k    = fx * ipd                          (once per frame)
 *   z    = depth, or far if depth is not a positive finite number
 *   zc   = min(max(z, near), far)            (the camera's near/far planes, Eq. 3)
 *   disp = k / zc
 *   t    = (x + 0.5) - disp
 *   xt   = floor(t)                          (the target pixel whose cell holds t)
 *
 * xt[y*w+x] receives the target column, or -1 if it falls outside [0, w).
 * zc[y*w+x] receives the clamped depth.
 */
void oracle_disparity(int w, int h, float fx, float ipd, float near_, float far_,
                      const float* depth, int32_t* xt, float* zc)
{
    const float k = fx * ipd;
#pragma omp parallel for schedule(static)
    for (int y = 0; y < h; ++y) {
        for (int x = 0; x < w; ++x) {
            size_t i = (size_t)y * (size_t)w + (size_t)x;
            float z = depth[i];
            if (!(z > 0.0f) || isinf(z)) z = far_;
            float c = fminf(fmaxf(z, near_), far_);
            float disp = k / c;
            float t = ((float)x + 0.5f) - disp;
            float f = floorf(t);
            xt[i] = (f >= 0.0f && f < (float)w) ? (int32_t)f : -1;
            zc[i] = c;
        }
    }
}

/*
 * Algorithm 2 (Reprojector stage 2), the write with the nearest kept.
 *
 * Each row is scanned left to right, as the per-row compute shader does; a source
 * pixel overwrites its target only if it is strictly nearer than what is there, so
 * on equal depth the first (lowest) source column keeps the target.  Smaller depth
 * is nearer (linear view-space z).
 *
 * The paper's scan also writes hole records into skipped pixels while it runs,
 * which makes the result depend on the scan order; here a hole is simply a target
 * that no source reaches, and its edges are found afterwards (oracle_hole_edges).
 *
 * src[y*w+u] receives the winning source column (same row, O1) or -1 for a hole;
 * zt[y*w+u] receives the winner's clamped depth, or +inf for a hole.
 */
void oracle_forward_warp(int w, int h, const int32_t* xt, const float* zc, int32_t* src, float* zt)
{
#pragma omp parallel for schedule(static)
    for (int y = 0; y < h; ++y) {
        for (int u = 0; u < w; ++u) {
            size_t i = (size_t)y * (size_t)w + (size_t)u;
            src[i] = -1;
            zt[i] = INFINITY;
        }
        for (int x = 0; x < w; ++x) {
            size_t i = (size_t)y * (size_t)w + (size_t)x;
            int t = xt[i];
            if (t < 0) continue;
            size_t o = (size_t)y * (size_t)w + (size_t)t;
            if (src[o] < 0 || zc[i] < zt[o]) {
                src[o] = x;
                zt[o] = zc[i];
            }
        }
    }
}

/*
 * Gather (Algorithm 3, non-hole branch): a reached target takes the source color of
 * the pixel that won it, all four bytes (alpha is carried like a color channel).
 * mask = 0 for reached targets and 1 for holes (disocclusions).  Hole pixels of
 * out_color are set to 0 here and written by oracle_fill.
 */
void oracle_resolve(int w, int h, const uint8_t* color, const int32_t* src, uint8_t* out_color,
                    uint8_t* mask)
{
#pragma omp parallel for schedule(static)
    for (int y = 0; y < h; ++y) {
        for (int u = 0; u < w; ++u) {
            size_t i = (size_t)y * (size_t)w + (size_t)u;
            if (src[i] >= 0) {
                size_t s = (size_t)y * (size_t)w + (size_t)src[i];
                memcpy(out_color + 4 * i, color + 4 * s, 4);
                mask[i] = 0;
            } else {
                memset(out_color + 4 * i, 0, 4);
                mask[i] = 1;
            }
        }
    }
}

/*
 * Disocclusion tracking (strategy (b)): for every hole pixel u of row y, the nearest
 * reached column on each side.  L = largest reached x < u (or -1), R = smallest
 * reached x > u (or w).  For reached pixels both are set to u.  In this frame L is
 * the occluder (foreground) side and R the background side of the hole; the hole
 * width of Algorithm 2 (target-column jump, edge to edge) is R - L.
 */
void oracle_hole_edges(int w, int h, const int32_t* src, int32_t* L, int32_t* R)
{
#pragma omp parallel for schedule(dynamic, 8)
    for (int y = 0; y < h; ++y) {
        const int32_t* s = src + (size_t)y * (size_t)w;
        for (int u = 0; u < w; ++u) {
            size_t i = (size_t)y * (size_t)w + (size_t)u;
            if (s[u] >= 0) {
                L[i] = u;
                R[i] = u;
                continue;
            }
            int l = u - 1;
            while (l >= 0 && s[l] < 0) --l;
            int r = u + 1;
            while (r < w && s[r] < 0) ++r;
            L[i] = l;
            R[i] = r;
        }
    }
}

/*
 * Patcher (Algorithm 3 with the weight of Eq. 6) for one hole pixel (v, u).
 *
 * Reading used (paper mirrored to a left-eye source):
 *   w      = R - L                       hole width of Algorithm 2
 *   d_occ  = zt(v, L), or 0 if L = -1    depth of the occluding edge
 *   t      = (R - u) / w                 Eq. 6's (u - r_x) / r_z, distance from the
 *                                        background edge over the hole width
 *   kernel = rows v-1, v, v+1 (h = 3, the paper's default height; rows outside the
 *            image skipped), and in each row the w + 1 columns from
 *            min(R + w, w_img - 1) down to R: the background side, farthest column
 *            first, as Algorithm 3's kernel runs from r.x - r.z up to r.x in the
 *            paper's frame.  Variants (Sec. Patcher: the kernel height is a
 *            parameter, 3 by default): kernel_rows = h gives rows v - (h-1)/2 .. v + (h-1)/2, and
 *            nearest_first visits each row's columns from R up instead.
 *   A candidate is skipped if it is a hole (it carries no color) or if it is
 *   strictly nearer than d_occ (a foreground pixel, observation O2).  Otherwise:
 *       wgt   = wrem / 2 + 0.3 wrem t   (Eq. 6, evaluated as (wrem * 0.5) +
 *                                        ((0.3 * wrem) * t), each step rounded)
 *       acc   = acc + C[j] * wgt         (per channel, multiply then add)
 *       wrem  = wrem - wgt
 *   Result: acc / (1 - wrem) per channel, rounded half to even and clamped to
 *   [0, 255].
 *   Fallback (no background edge, R = w_img, or no candidate contributed): copy the
 *   warped color at (v, R) if R < w_img, else at (v, L) if L >= 0, else zero.
 */
static void fill_one(int w, int h, int v, int u, int L, int R, const int32_t* src, const float* zt,
                     const uint8_t* warped, int kernel_rows, int nearest_first, uint8_t out[4])
{
    if (R < w) {
        int wd = R - L;
        float d_occ = (L >= 0) ? zt[(size_t)v * (size_t)w + (size_t)L] : 0.0f;
        float t = (float)(R - u) / (float)wd;
        float acc[4] = { 0.0f, 0.0f, 0.0f, 0.0f };
        float wrem = 1.0f;
        int hr = (kernel_rows - 1) / 2;
        int jhi = R + wd;
        if (jhi > w - 1) jhi = w - 1;
        for (int vv = v - hr; vv <= v + hr; ++vv) {
            if (vv < 0 || vv >= h) continue;
            for (int s = 0; s <= jhi - R; ++s) {
                int j = nearest_first ? R + s : jhi - s;
                size_t q = (size_t)vv * (size_t)w + (size_t)j;
                if (src[q] < 0) continue;
                if (zt[q] < d_occ) continue;
                float a = wrem * 0.5f;
                float b = (0.3f * wrem) * t;
                float wgt = a + b;
                for (int c = 0; c < 4; ++c) {
                    float term = (float)warped[4 * q + c] * wgt;
                    acc[c] = acc[c] + term;
                }
                wrem = wrem - wgt;
            }
        }
        if (wrem != 1.0f) {
            float den = 1.0f - wrem;
            for (int c = 0; c < 4; ++c) {
                float r = rintf(acc[c] / den);
                if (r < 0.0f) r = 0.0f;
                if (r > 255.0f) r = 255.0f;
                out[c] = (uint8_t)r;
            }
            return;
        }
    }
    if (R < w)
        memcpy(out, warped + 4 * ((size_t)v * (size_t)w + (size_t)R), 4);
    else if (L >= 0)
        memcpy(out, warped + 4 * ((size_t)v * (size_t)w + (size_t)L), 4);
    else
        memset(out, 0, 4);
}

/*
 * Fill every hole pixel (mask = 1) of `warped` (the resolved image) into out_color;
 * reached pixels are copied unchanged.  Candidates are read from `warped` only.
 * kernel_rows is the kernel height h of the Patcher (odd, >= 1; the paper's default
 * is 3): rows v - (h-1)/2 .. v + (h-1)/2.  nearest_first = 0 visits each row's columns
 * from the farthest, min(R + w, W - 1), down to R (the paper's order, mirrored);
 * nearest_first = 1 visits them from R up.
 */
void oracle_fill_ex(int w, int h, const int32_t* src, const float* zt, const int32_t* L, const int32_t* R,
                    const uint8_t* warped, int kernel_rows, int nearest_first, uint8_t* out_color)
{
#pragma omp parallel for schedule(dynamic, 4)
    for (int v = 0; v < h; ++v) {
        for (int u = 0; u < w; ++u) {
            size_t i = (size_t)v * (size_t)w + (size_t)u;
            if (src[i] >= 0) {
                memcpy(out_color + 4 * i, warped + 4 * i, 4);
                continue;
            }
            fill_one(w, h, v, u, L[i], R[i], src, zt, warped, kernel_rows, nearest_first, out_color + 4 * i);
        }
    }
}

void oracle_fill(int w, int h, const int32_t* src, const float* zt, const int32_t* L, const int32_t* R,
                 const uint8_t* warped, uint8_t* out_color)
{
    oracle_fill_ex(w, h, src, zt, L, R, warped, 3, 0, out_color);
}

/*
 * The whole path, left eye -> right eye.  fy, cx and cy are accepted for the
 * camera description but do not enter the result: for a parallel-axis pair with
 * shared intrinsics the vertical coordinate is unchanged and cx cancels.
 * Returns 0, -1 on bad sizes, -2 if a temporary could not be allocated.
 */
int oracle_synthesize_ex(int w, int h, float fx, float fy, float cx, float cy, float ipd, float near_,
                         float far_, const uint8_t* color, const float* depth, int kernel_rows, int nearest_first,
                         uint8_t* out_color, uint8_t* mask)
{
    (void)fy;
    (void)cx;
    (void)cy;
    if (w < 0 || h < 0 || kernel_rows < 1 || (kernel_rows & 1) == 0) return -1;
    size_t n = (size_t)w * (size_t)h;
    if (n == 0) return 0;
    int32_t* xt = (int32_t*)malloc(n * sizeof(int32_t));
    float* zc = (float*)malloc(n * sizeof(float));
    int32_t* src = (int32_t*)malloc(n * sizeof(int32_t));
    float* zt = (float*)malloc(n * sizeof(float));
    int32_t* L = (int32_t*)malloc(n * sizeof(int32_t));
    int32_t* R = (int32_t*)malloc(n * sizeof(int32_t));
    uint8_t* warped = (uint8_t*)malloc(n * 4);
    int rc = 0;
    if (!xt || !zc || !src || !zt || !L || !R || !warped) {
        rc = -2;
    } else {
        oracle_disparity(w, h, fx, ipd, near_, far_, depth, xt, zc);
        oracle_forward_warp(w, h, xt, zc, src, zt);
        oracle_resolve(w, h, color, src, warped, mask);
        oracle_hole_edges(w, h, src, L, R);
        oracle_fill_ex(w, h, src, zt, L, R, warped, kernel_rows, nearest_first, out_color);
    }
    free(xt);
    free(zc);
    free(src);
    free(zt);
    free(L);
    free(R);
    free(warped);
    return rc;
}

int oracle_synthesize(int w, int h, float fx, float fy, float cx, float cy, float ipd, float near_,
                      float far_, const uint8_t* color, const float* depth, uint8_t* out_color,
                      uint8_t* mask)
{
    return oracle_synthesize_ex(w, h, fx, fy, cx, cy, ipd, near_, far_, color, depth, 3, 0, out_color, mask);
}

/*
 * Strategies (c) and (d) of the Reprojector: the resolution-independent intermediate
 * buffer (ImBuffer) downsampled along the row, and the optional linear interpolation.
 * The paper gives only their intent (the buffer keeps how far each pixel moves along
 * its row, the full-resolution image is sampled at a linearly interpolated shift, and a
 * reached pixel takes its color from the rendered image at the position the buffer
 * gives); the reading written out here:
 *
 *   s = div in {1, 2, 4, 8, 16} (1/2 .. 1/16 of the per-eye resolution, along the row:
 *   the warp moves pixels along rows only, O1, so rows stay at full resolution).
 *   Row y has ws = ceil(w / s) cells; cell i stands for source pixels s i .. s i + s - 1.
 *
 *   1. Algorithm 1 per cell, on its representative pixel p = min(s i + s/2, w - 1):
 *      zc = clamp(depth(y, p)) as in oracle_disparity, disp = k / zc,
 *      t = (p + 0.5) - disp, target cell floor(t / s) (dropped outside [0, ws)).
 *   2. Algorithm 2 per row over the cells: nearest kept, the first on equal depth.
 *      A target cell records its winner's cell i, zc and disp (the shift).
 *   3. Full resolution: pixel x lies in cell j = floor(x / s); it is a hole if that
 *      cell is, otherwise its depth is the winner's zc and its color
 *        interp = 0: the source pixel at the same place in the winning cell,
 *                    min(s i + (x - s j), w - 1);
 *        interp = 1: the shift D linearly between cell j's and the neighbouring cell's
 *                    on the side of the pixel centre x + 0.5 (weight |x + 0.5 - c_j| / s
 *                    with c_j = s j + s/2 the cell centre; D = disp_j if that neighbour is
 *                    a hole or outside the row); the color sampled at texel coordinate
 *                    u = x + D (texel centres at integers): clamped to the row's first or
 *                    last texel outside [0, w - 1], otherwise c0 + (c1 - c0) f between the
 *                    texels floor(u) and floor(u) + 1 with f = u - floor(u), per channel,
 *                    rounded half to even.
 *   4. Algorithm 3 with Eq. 6 at full resolution over that image (oracle_hole_edges,
 *      oracle_fill_ex), its reached pixels the candidates.
 *
 * With s = 1 and interp = 0 every step is the base path's, so the result equals
 * oracle_synthesize_ex's.  Returns 0, -1 on bad arguments, -2 if a temporary could
 * not be allocated.
 */
int oracle_synthesize_imb(int w, int h, float fx, float ipd, float near_, float far_, const uint8_t* color,
                          const float* depth, int div, int interp, int kernel_rows, int nearest_first,
                          uint8_t* out_color, uint8_t* mask)
{
    if (w < 0 || h < 0 || kernel_rows < 1 || (kernel_rows & 1) == 0) return -1;
    if (div != 1 && div != 2 && div != 4 && div != 8 && div != 16) return -1;
    if (interp != 0 && interp != 1) return -1;
    size_t n = (size_t)w * (size_t)h;
    if (n == 0) return 0;
    const int ws = (w + div - 1) / div;
    const float k = fx * ipd;
    const size_t nc = (size_t)ws * (size_t)h;
    int32_t* win = (int32_t*)malloc(nc * sizeof(int32_t));  /* winner cell, or -1 */
    float* wz = (float*)malloc(nc * sizeof(float));        /* winner's zc */
    float* wd = (float*)malloc(nc * sizeof(float));        /* winner's disp */
    int32_t* src = (int32_t*)malloc(n * sizeof(int32_t));  /* full resolution: >= 0 reached */
    float* zt = (float*)malloc(n * sizeof(float));
    int32_t* L = (int32_t*)malloc(n * sizeof(int32_t));
    int32_t* R = (int32_t*)malloc(n * sizeof(int32_t));
    uint8_t* warped = (uint8_t*)malloc(n * 4);
    int rc = 0;
    if (!win || !wz || !wd || !src || !zt || !L || !R || !warped) {
        rc = -2;
        goto done;
    }
    for (int y = 0; y < h; ++y) {
        int32_t* wrow = win + (size_t)y * (size_t)ws;
        float* zrow = wz + (size_t)y * (size_t)ws;
        float* drow = wd + (size_t)y * (size_t)ws;
        for (int j = 0; j < ws; ++j) wrow[j] = -1;
        /* steps 1 and 2: the cells of the row, scanned left to right */
        for (int i = 0; i < ws; ++i) {
            int p = div * i + div / 2;
            if (p > w - 1) p = w - 1;
            float z = depth[(size_t)y * (size_t)w + (size_t)p];
            if (!(z > 0.0f) || isinf(z)) z = far_;
            float c = fminf(fmaxf(z, near_), far_);
            float disp = k / c;
            float t = ((float)p + 0.5f) - disp;
            float tc = floorf(t / (float)div);
            if (!(tc >= 0.0f && tc < (float)ws)) continue;
            int j = (int)tc;
            if (wrow[j] < 0 || c < zrow[j]) {
                wrow[j] = i;
                zrow[j] = c;
                drow[j] = disp;
            }
        }
        /* step 3: full resolution */
        for (int x = 0; x < w; ++x) {
            size_t q = (size_t)y * (size_t)w + (size_t)x;
            int j = x / div;
            if (wrow[j] < 0) {
                src[q] = -1;
                zt[q] = INFINITY;
                memset(warped + 4 * q, 0, 4);
                mask[q] = 1;
                continue;
            }
            src[q] = 0;
            zt[q] = zrow[j];
            mask[q] = 0;
            const uint8_t* crow = color + 4 * (size_t)y * (size_t)w;
            if (!interp) {
                int sx = div * wrow[j] + (x - div * j);
                if (sx > w - 1) sx = w - 1;
                memcpy(warped + 4 * q, crow + 4 * (size_t)sx, 4);
                continue;
            }
            float centre = (float)(div * j) + 0.5f * (float)div;
            float off = ((float)x + 0.5f) - centre;
            int nb = off < 0.0f ? j - 1 : j + 1;
            float D = drow[j];
            if (off != 0.0f && nb >= 0 && nb < ws && wrow[nb] >= 0) {
                float a = fabsf(off) / (float)div;
                D = drow[j] + (drow[nb] - drow[j]) * a;
            }
            float u = (float)x + D;
            if (u <= 0.0f) {
                memcpy(warped + 4 * q, crow, 4);
            } else if (u >= (float)(w - 1)) {
                memcpy(warped + 4 * q, crow + 4 * (size_t)(w - 1), 4);
            } else {
                float fl = floorf(u);
                int i0 = (int)fl;
                float f = u - fl;
                for (int ch = 0; ch < 4; ++ch) {
                    float c0 = (float)crow[4 * (size_t)i0 + ch];
                    float c1 = (float)crow[4 * (size_t)(i0 + 1) + ch];
                    float v = c0 + (c1 - c0) * f;
                    warped[4 * q + ch] = (uint8_t)rintf(v);
                }
            }
        }
    }
    /* step 4 */
    oracle_hole_edges(w, h, src, L, R);
    oracle_fill_ex(w, h, src, zt, L, R, warped, kernel_rows, nearest_first, out_color);
done:
    free(win);
    free(wz);
    free(wd);
    free(src);
    free(zt);
    free(L);
    free(R);
    free(warped);
    return rc;
}

/*
 * General reprojection (Eq. 5 with a general M = (VP_left)^-1 VP_right): the second eye
 * may be rotated and offset in any direction, so a pixel can leave its row.  Reading:
 * both eyes share the pinhole intrinsics (fx, fy, cx, cy); the second eye sits at
 * position c (left-eye camera coordinates) with rotation rot (row-major 3x3, mapping
 * left-eye camera axes to the second eye's: p' = rot (p - c)).
 *
 *   1. Per source pixel (y, x): zc = clamp(depth) as in oracle_disparity (Alg. 1);
 *      P = ((x + 0.5 - cx) zc / fx, (y + 0.5 - cy) zc / fy, zc);
 *      P' = rot (P - c), each row as ((r0 q0 + r1 q1) + r2 q2);
 *      dropped unless P'.z > 0; target (floor(fx P'.x / P'.z + cx),
 *      floor(fy P'.y / P'.z + cy)), dropped outside the frame.
 *   2. Alg. 2 per target pixel over the whole frame: the nearest P'.z kept, the lower
 *      source index y w + x on equal depth (the first of a row-major scan).
 *   3. Gather the winner's color; its P'.z is the target's depth.
 *   4. Holes along each row and the Patcher (oracle_hole_edges, oracle_fill_ex), the
 *      candidates' depths being the targets' P'.z.
 *
 * With rot = I and c = (ipd, 0, 0) the target row is y and the column is the base
 * path's up to rounding; for dyadic parameters (powers of two for fx and the depths,
 * integers for cx) every step is exact and the result equals oracle_synthesize_ex's.
 * Returns 0, -1 on bad arguments, -2 if a temporary could not be allocated.
 */
int oracle_synthesize_pose(int w, int h, float fx, float fy, float cx, float cy, const float* rot, const float* c,
                           float near_, float far_, const uint8_t* color, const float* depth, int kernel_rows,
                           int nearest_first, uint8_t* out_color, uint8_t* mask)
{
    if (w < 0 || h < 0 || kernel_rows < 1 || (kernel_rows & 1) == 0) return -1;
    size_t n = (size_t)w * (size_t)h;
    if (n == 0) return 0;
    int64_t* win = (int64_t*)malloc(n * sizeof(int64_t));  /* winner source index, or -1 */
    float* zt = (float*)malloc(n * sizeof(float));
    int32_t* src = (int32_t*)malloc(n * sizeof(int32_t));
    int32_t* L = (int32_t*)malloc(n * sizeof(int32_t));
    int32_t* R = (int32_t*)malloc(n * sizeof(int32_t));
    uint8_t* warped = (uint8_t*)malloc(n * 4);
    int rc = 0;
    if (!win || !zt || !src || !L || !R || !warped) {
        rc = -2;
        goto done;
    }
    for (size_t i = 0; i < n; ++i) {
        win[i] = -1;
        zt[i] = INFINITY;
    }
    /* steps 1 and 2: a row-major scan of the sources */
    for (int y = 0; y < h; ++y) {
        for (int x = 0; x < w; ++x) {
            size_t i = (size_t)y * (size_t)w + (size_t)x;
            float z = depth[i];
            if (!(z > 0.0f) || isinf(z)) z = far_;
            float zc = fminf(fmaxf(z, near_), far_);
            float px = (((float)x + 0.5f) - cx) * zc / fx;
            float py = (((float)y + 0.5f) - cy) * zc / fy;
            float q0 = px - c[0], q1 = py - c[1], q2 = zc - c[2];
            float X = (rot[0] * q0 + rot[1] * q1) + rot[2] * q2;
            float Y = (rot[3] * q0 + rot[4] * q1) + rot[5] * q2;
            float Z = (rot[6] * q0 + rot[7] * q1) + rot[8] * q2;
            if (!(Z > 0.0f)) continue;
            float u = floorf(fx * X / Z + cx);
            float v = floorf(fy * Y / Z + cy);
            if (!(u >= 0.0f && u < (float)w && v >= 0.0f && v < (float)h)) continue;
            size_t o = (size_t)v * (size_t)w + (size_t)u;
            if (win[o] < 0 || Z < zt[o]) {
                win[o] = (int64_t)i;
                zt[o] = Z;
            }
        }
    }
    /* step 3 */
    for (size_t o = 0; o < n; ++o) {
        if (win[o] >= 0) {
            memcpy(warped + 4 * o, color + 4 * (size_t)win[o], 4);
            src[o] = 0;
            mask[o] = 0;
        } else {
            memset(warped + 4 * o, 0, 4);
            src[o] = -1;
            mask[o] = 1;
        }
    }
    /* step 4 */
    oracle_hole_edges(w, h, src, L, R);
    oracle_fill_ex(w, h, src, zt, L, R, warped, kernel_rows, nearest_first, out_color);
done:
    free(win);
    free(zt);
    free(src);
    free(L);
    free(R);
    free(warped);
    return rc;
}
