/*
 * Seeded synthetic scenes and an analytic ray caster (host C, input generation only).
 *
 * This module produces the inputs of second-eye synthesis: a rendered eye's RGBA8
 * color and FP32 linear view-space depth (plus a primitive id per pixel, for tests).
 * It stands in for the renderer of the method's system overview (Sec. "System
 * Overview": render once for the dominant eye, keep the RGB and depth G-buffers,
 * Sec. "G-Buffers Exploration").  It holds none of the synthesis arithmetic: no
 * disparity, warp or fill.  The same code renders the right eye from its own
 * position, which gives the analytic ground truth of the second eye.
 *
 * Camera: pinhole at (eye_x, 0, 0) looking down +z, image y pointing down, world y
 * up.  The ray through the centre of pixel (x, y) is
 *     d = ((x + 0.5 - cx) / fx, -(y + 0.5 - cy) / fy, 1),
 * so the ray parameter of a hit equals its view-space depth z.
 *
 * Scene: n_prims spheres or axis-aligned boxes (probability 1/2 each).  For each,
 * a front depth d (uniform or log-uniform in [zmin, zmax]) and a size r (uniform
 * in [rmin, rmax]) are drawn; the centre sits at depth d + r (sphere) or d + hz
 * (box), so no geometry is nearer than d and both eyes (at z = 0) are outside
 * every primitive.  The centre's x and y are uniform across the view frustum at
 * that depth.  Optional ground plane y = ground_y with a 1 m checker albedo.
 * Lambert shading, one directional light, ambient 0.1; misses get the sky color
 * and depth = far.  All random draws come from splitmix64 over (seed, counter),
 * so a scene is a pure function of (cfg, seed).
 *
 * Work is split over host threads by 16x16 tiles; each tile tests only the
 * primitives whose conservative screen rectangle overlaps it, in index order, so
 * the output does not depend on the thread count.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <unistd.h>

typedef struct {
    int32_t w, h;
    int32_t n_prims;
    int32_t ground;     /* 1: ground plane at y = ground_y                 */
    int32_t log_depth;  /* 1: front depth log-uniform, 0: uniform          */
    float zmin, zmax;   /* front-depth range of the primitives (m)         */
    float rmin, rmax;   /* size range (m)                                  */
    float fx, fy, cx, cy;
    float far_;         /* depth written for rays that hit nothing         */
    float ground_y;
    float max_cover;    /* >0: redraw a primitive whose screen rectangle covers more than
                           this fraction of the image (left eye)                       */
} scene_cfg;

enum { PRIM_SPHERE = 0, PRIM_BOX = 1 };

typedef struct {
    int type;
    double c[3];    /* centre                                  */
    double r;       /* sphere radius                           */
    double he[3];   /* box half extents                        */
    double albedo[3];
} prim_t;

#define TILE 16

static uint64_t splitmix64(uint64_t x)
{
    x += 0x9E3779B97F4A7C15ull;
    x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
    x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
    return x ^ (x >> 31);
}

typedef struct { uint64_t seed, ctr; } rng_t;

static double rng_u01(rng_t* g)
{
    uint64_t v = splitmix64(g->seed * 0x2545F4914F6CDD1Dull + (g->ctr++));
    return (double)(v >> 11) * (1.0 / 9007199254740992.0);
}

static void prim_rect(const scene_cfg* cfg, const prim_t* q, double eye_x, int r[4]);

/* Draw one primitive (type, size, front depth, frustum position, albedo). */
static void draw_prim(const scene_cfg* cfg, rng_t* g, prim_t* q)
{
    q->type = rng_u01(g) < 0.5 ? PRIM_SPHERE : PRIM_BOX;
    double r = cfg->rmin + rng_u01(g) * (cfg->rmax - cfg->rmin);
    double u = rng_u01(g);
    double d;
    if (cfg->log_depth)
        d = exp(log((double)cfg->zmin) + u * (log((double)cfg->zmax) - log((double)cfg->zmin)));
    else
        d = cfg->zmin + u * (cfg->zmax - cfg->zmin);
    double hz = r;
    if (q->type == PRIM_BOX) {
        q->he[0] = r * (0.5 + 0.5 * rng_u01(g));
        q->he[1] = r * (0.5 + 0.5 * rng_u01(g));
        q->he[2] = r * (0.5 + 0.5 * rng_u01(g));
        hz = q->he[2];
    } else {
        q->he[0] = q->he[1] = q->he[2] = r;
    }
    q->r = r;
    double cz = d + hz;
    double sx = (2.0 * rng_u01(g) - 1.0) * (0.5 * cfg->w / cfg->fx);
    double sy = (2.0 * rng_u01(g) - 1.0) * (0.5 * cfg->h / cfg->fy);
    q->c[0] = sx * cz;
    q->c[1] = sy * cz;
    q->c[2] = cz;
    for (int k = 0; k < 3; ++k) q->albedo[k] = 0.2 + 0.8 * rng_u01(g);
}

/*
 * A primitive is redrawn (up to 10000 times) while its conservative screen rectangle
 * covers more than max_cover of the image, so that no single near primitive fills the
 * view.  The proposal distributions are the configured ones.
 */
static void make_scene(const scene_cfg* cfg, uint64_t seed, prim_t* p)
{
    rng_t g = { seed + 1, 0 };
    for (int i = 0; i < cfg->n_prims; ++i) {
        for (int attempt = 0; attempt < 10000; ++attempt) {
            draw_prim(cfg, &g, &p[i]);
            if (!(cfg->max_cover > 0.0f)) break;
            int r[4];
            prim_rect(cfg, &p[i], 0.0, r);
            double x0 = r[0] < 0 ? 0 : r[0], x1 = r[1] >= cfg->w ? cfg->w - 1 : r[1];
            double y0 = r[2] < 0 ? 0 : r[2], y1 = r[3] >= cfg->h ? cfg->h - 1 : r[3];
            double area = (x1 >= x0 && y1 >= y0) ? (x1 - x0 + 1) * (y1 - y0 + 1) : 0.0;
            if (area <= cfg->max_cover * (double)cfg->w * (double)cfg->h) break;
        }
    }
}

/* Ray-primitive hit: returns the ray parameter s > 0 of the first hit (or +inf) and its normal. */
static double hit_sphere(const prim_t* q, const double o[3], const double d[3], double n[3])
{
    double oc[3] = { o[0] - q->c[0], o[1] - q->c[1], o[2] - q->c[2] };
    double a = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
    double b = oc[0] * d[0] + oc[1] * d[1] + oc[2] * d[2];
    double cc = oc[0] * oc[0] + oc[1] * oc[1] + oc[2] * oc[2] - q->r * q->r;
    double disc = b * b - a * cc;
    if (disc < 0.0) return INFINITY;
    double s = (-b - sqrt(disc)) / a;
    if (!(s > 0.0)) return INFINITY;
    for (int k = 0; k < 3; ++k) n[k] = (o[k] + s * d[k] - q->c[k]) / q->r;
    return s;
}

static double hit_box(const prim_t* q, const double o[3], const double d[3], double n[3])
{
    double tnear = -INFINITY, tfar = INFINITY;
    int axis = 0;
    double sgn = 1.0;
    for (int k = 0; k < 3; ++k) {
        double lo = q->c[k] - q->he[k], hi = q->c[k] + q->he[k];
        if (d[k] == 0.0) {
            if (o[k] < lo || o[k] > hi) return INFINITY;
            continue;
        }
        double t1 = (lo - o[k]) / d[k], t2 = (hi - o[k]) / d[k];
        double s1 = -1.0;
        if (t1 > t2) { double tt = t1; t1 = t2; t2 = tt; s1 = 1.0; }
        if (t1 > tnear) { tnear = t1; axis = k; sgn = s1; }
        if (t2 < tfar) tfar = t2;
    }
    if (!(tnear <= tfar) || !(tnear > 0.0)) return INFINITY;
    n[0] = n[1] = n[2] = 0.0;
    n[axis] = sgn;
    return tnear;
}

static uint8_t to_u8(double v)
{
    double s = 255.0 * v;
    if (s < 0.0) s = 0.0;
    if (s > 255.0) s = 255.0;
    return (uint8_t)lrint(s);
}

typedef struct {
    const scene_cfg* cfg;
    const prim_t* prims;
    double eye_x;
    int tiles_x, tiles_y;
    const int32_t* tile_off;   /* CSR over tiles */
    const int32_t* tile_list;
    uint8_t* color;
    float* depth;
    int32_t* prim_id;
    int next_tile_row;
    pthread_mutex_t lock;
} job_t;

static const double LIGHT[3] = { -0.3713906763541037, 0.7427813527082074, -0.5570860145311556 };
static const uint8_t SKY[4] = { 110, 160, 230, 255 };

static void shade_pixel(job_t* J, int x, int y)
{
    const scene_cfg* cfg = J->cfg;
    double o[3] = { J->eye_x, 0.0, 0.0 };
    double d[3] = { (x + 0.5 - cfg->cx) / cfg->fx, -((y + 0.5 - cfg->cy) / cfg->fy), 1.0 };
    int tile = (y / TILE) * J->tiles_x + (x / TILE);
    double best = INFINITY, bn[3] = { 0, 0, 0 };
    int best_id = -1;
    for (int e = J->tile_off[tile]; e < J->tile_off[tile + 1]; ++e) {
        int i = J->tile_list[e];
        double n[3];
        double s = J->prims[i].type == PRIM_SPHERE ? hit_sphere(&J->prims[i], o, d, n)
                                                   : hit_box(&J->prims[i], o, d, n);
        if (s < best) { best = s; best_id = i; bn[0] = n[0]; bn[1] = n[1]; bn[2] = n[2]; }
    }
    double alb[3];
    if (cfg->ground && d[1] < 0.0) {
        double s = cfg->ground_y / d[1];
        if (s > 0.0 && s < best) {
            best = s;
            best_id = cfg->n_prims;
            bn[0] = 0.0; bn[1] = 1.0; bn[2] = 0.0;
        }
    }
    size_t idx = (size_t)y * cfg->w + x;
    if (best_id < 0 || !(best <= (double)cfg->far_)) {
        memcpy(J->color + 4 * idx, SKY, 4);
        J->depth[idx] = cfg->far_;
        J->prim_id[idx] = -1;
        return;
    }
    if (best_id == cfg->n_prims) {
        double gx = o[0] + best * d[0], gz = o[2] + best * d[2];
        int chk = ((int)floor(gx) + (int)floor(gz)) & 1;
        alb[0] = chk ? 0.75 : 0.40;
        alb[1] = chk ? 0.72 : 0.42;
        alb[2] = chk ? 0.65 : 0.38;
    } else {
        alb[0] = J->prims[best_id].albedo[0];
        alb[1] = J->prims[best_id].albedo[1];
        alb[2] = J->prims[best_id].albedo[2];
    }
    double ndl = bn[0] * LIGHT[0] + bn[1] * LIGHT[1] + bn[2] * LIGHT[2];
    double sh = 0.1 + 0.9 * (ndl > 0.0 ? ndl : 0.0);
    J->color[4 * idx + 0] = to_u8(alb[0] * sh);
    J->color[4 * idx + 1] = to_u8(alb[1] * sh);
    J->color[4 * idx + 2] = to_u8(alb[2] * sh);
    J->color[4 * idx + 3] = 255;
    J->depth[idx] = (float)best;
    J->prim_id[idx] = best_id;
}

static void* worker(void* arg)
{
    job_t* J = (job_t*)arg;
    for (;;) {
        pthread_mutex_lock(&J->lock);
        int ty = J->next_tile_row++;
        pthread_mutex_unlock(&J->lock);
        if (ty >= J->tiles_y) break;
        int y0 = ty * TILE, y1 = y0 + TILE < J->cfg->h ? y0 + TILE : J->cfg->h;
        for (int y = y0; y < y1; ++y)
            for (int x = 0; x < J->cfg->w; ++x) shade_pixel(J, x, y);
    }
    return NULL;
}

/* Conservative pixel rectangle of a primitive's AABB seen from (eye_x, 0, 0). */
static void prim_rect(const scene_cfg* cfg, const prim_t* q, double eye_x, int r[4])
{
    double umin = INFINITY, umax = -INFINITY, vmin = INFINITY, vmax = -INFINITY;
    for (int c = 0; c < 8; ++c) {
        double X = q->c[0] + ((c & 1) ? q->he[0] : -q->he[0]) - eye_x;
        double Y = q->c[1] + ((c & 2) ? q->he[1] : -q->he[1]);
        double Z = q->c[2] + ((c & 4) ? q->he[2] : -q->he[2]);
        double u = cfg->fx * X / Z + cfg->cx;
        double v = -cfg->fy * Y / Z + cfg->cy;
        if (u < umin) umin = u;
        if (u > umax) umax = u;
        if (v < vmin) vmin = v;
        if (v > vmax) vmax = v;
    }
    double lim = 4.0 * (cfg->w + cfg->h);
    if (umin < -lim) umin = -lim;
    if (vmin < -lim) vmin = -lim;
    if (umax > lim) umax = lim;
    if (vmax > lim) vmax = lim;
    r[0] = (int)floor(umin) - 2;
    r[1] = (int)ceil(umax) + 2;
    r[2] = (int)floor(vmin) - 2;
    r[3] = (int)ceil(vmax) + 2;
}

/*
 * Render one eye of scene (cfg, seed) from (eye_x, 0, 0).
 * color: h*w*4 bytes, depth: h*w floats, prim_id: h*w int32 (-1 sky, n_prims ground).
 * Returns 0, or -1 on bad arguments / allocation failure.
 */
int scene_render(const scene_cfg* cfg, uint64_t seed, float eye_x, uint8_t* color, float* depth,
                 int32_t* prim_id, int nthreads)
{
    if (!cfg || cfg->w <= 0 || cfg->h <= 0 || cfg->n_prims < 0 || !color || !depth || !prim_id) return -1;
    prim_t* prims = (prim_t*)calloc(cfg->n_prims > 0 ? cfg->n_prims : 1, sizeof(prim_t));
    if (!prims) return -1;
    make_scene(cfg, seed, prims);
    int tx = (cfg->w + TILE - 1) / TILE, ty = (cfg->h + TILE - 1) / TILE;
    int32_t* off = (int32_t*)calloc((size_t)tx * ty + 1, sizeof(int32_t));
    int (*rects)[4] = (int (*)[4])calloc(cfg->n_prims > 0 ? cfg->n_prims : 1, sizeof(int[4]));
    if (!off || !rects) { free(prims); free(off); free(rects); return -1; }
    for (int i = 0; i < cfg->n_prims; ++i) {
        prim_rect(cfg, &prims[i], eye_x, rects[i]);
        int x0 = rects[i][0] < 0 ? 0 : rects[i][0] / TILE;
        int x1 = rects[i][1] >= cfg->w ? tx - 1 : rects[i][1] / TILE;
        int y0 = rects[i][2] < 0 ? 0 : rects[i][2] / TILE;
        int y1 = rects[i][3] >= cfg->h ? ty - 1 : rects[i][3] / TILE;
        if (rects[i][1] < 0 || rects[i][3] < 0 || rects[i][0] >= cfg->w || rects[i][2] >= cfg->h) {
            rects[i][0] = 1; rects[i][1] = 0; /* empty */
            continue;
        }
        rects[i][0] = x0; rects[i][1] = x1; rects[i][2] = y0; rects[i][3] = y1;
        for (int b = y0; b <= y1; ++b)
            for (int a = x0; a <= x1; ++a) off[b * tx + a + 1]++;
    }
    for (int t = 0; t < tx * ty; ++t) off[t + 1] += off[t];
    int32_t* list = (int32_t*)malloc(((size_t)off[tx * ty] + 1) * sizeof(int32_t));
    int32_t* fill = (int32_t*)calloc((size_t)tx * ty, sizeof(int32_t));
    if (!list || !fill) { free(prims); free(off); free(rects); free(list); free(fill); return -1; }
    for (int i = 0; i < cfg->n_prims; ++i) {
        if (rects[i][0] > rects[i][1]) continue;
        for (int b = rects[i][2]; b <= rects[i][3]; ++b)
            for (int a = rects[i][0]; a <= rects[i][1]; ++a) {
                int t = b * tx + a;
                list[off[t] + fill[t]++] = i;
            }
    }
    job_t J;
    J.cfg = cfg; J.prims = prims; J.eye_x = eye_x; J.tiles_x = tx; J.tiles_y = ty;
    J.tile_off = off; J.tile_list = list; J.color = color; J.depth = depth; J.prim_id = prim_id;
    J.next_tile_row = 0;
    pthread_mutex_init(&J.lock, NULL);
    if (nthreads <= 0) {
        long n = sysconf(_SC_NPROCESSORS_ONLN);
        nthreads = n > 0 ? (int)n : 1;
    }
    if (nthreads > 64) nthreads = 64;
    pthread_t th[64];
    int started = 0;
    for (int i = 1; i < nthreads; ++i)
        if (pthread_create(&th[started], NULL, worker, &J) == 0) started++;
    worker(&J);
    for (int i = 0; i < started; ++i) pthread_join(th[i], NULL);
    pthread_mutex_destroy(&J.lock);
    free(prims); free(off); free(rects); free(list); free(fill);
    return 0;
}
