// C ABI of the second-eye synthesis library: argument checks, dispatch, ownership.
// Declarations and the contract of every entry point are in include/yoro.h.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <utility>
#include <vector>

#include "yoro.h"
#include "yoro_internal.h"

using yoro::FrameArgs;
using yoro::FusedLimits;

struct yoro_ctx {
    int w, h;
    float fx, fy, cx, cy, ipd, near_, far_;
    float k;
    int device;
    int halo, nearest;  // Patcher kernel shape (yoro_options)
    int imb_div, imb_interp;  // row-downsampled intermediate buffer (yoro_create_imb)
    bool pose;                // general second-eye pose (yoro_create_pose)
    yoro::PoseArgs pose_args; // its camera and pose (scratch pointers bound per call)
    bool fused_ok;      // the window of one band row fits shared memory
    FusedLimits lim;
    yoro::FusedShape shape;
    unsigned long long* d_zbuf;    // unfused path, h*w keys, allocated on first use
    unsigned char* d_stage;        // host-buffer path, 13*h*w bytes (+ padding), on first use
    void* d_imb;                   // intermediate-buffer path: cell keys and depths, on first use
    void* d_pose;                  // general-pose path: keys and depths, on first use
};

namespace {

thread_local yoro_status g_last_create = YORO_OK;

bool finite_all(std::initializer_list<float> v)
{
    for (float x : v)
        if (!std::isfinite(x)) return false;
    return true;
}

bool camera_ok(int w, int h, float fx, float fy, float cx, float cy, float ipd, float near_, float far_)
{
    if (w < 0 || h < 0) return false;
    if ((int64_t)w * (int64_t)h >= ((int64_t)1 << 31)) return false;
    if (!finite_all({fx, fy, cx, cy, ipd, near_, far_})) return false;
    if (!(fx > 0.0f) || !(ipd >= 0.0f) || !(near_ > 0.0f) || !(far_ > near_)) return false;
    return true;
}

bool aligned(const void* p, uintptr_t a) { return ((uintptr_t)p & (a - 1)) == 0; }

bool overlaps(const void* a, size_t na, const void* b, size_t nb)
{
    const uintptr_t x = (uintptr_t)a, y = (uintptr_t)b;
    return x < y + nb && y < x + na;
}

// Checks shared by every device-pointer entry point.  Fills `f` on success.
yoro_status make_frame(int w, int h, float k, float near_, float far_, const void* color, const float* depth,
                       void* out, unsigned char* mask, FrameArgs* f)
{
    const size_t n = (size_t)w * (size_t)h;
    if (!color || !depth || !out || !mask) return YORO_EINVAL;
    if (!aligned(color, 4) || !aligned(depth, 4) || !aligned(out, 4)) return YORO_EALIGN;
    if (overlaps(out, 4 * n, color, 4 * n) || overlaps(out, 4 * n, depth, 4 * n) ||
        overlaps(mask, n, color, 4 * n) || overlaps(mask, n, depth, 4 * n) || overlaps(mask, n, out, 4 * n))
        return YORO_EINVAL;
    f->color = (const uint32_t*)color;
    f->depth = depth;
    f->out = (uint32_t*)out;
    f->mask = mask;
    f->w = w;
    f->h = h;
    f->k = k;
    f->near_ = near_;
    f->far_ = far_;
    // M bounds 2^-20 (xc + q + 1) over the frame: xc <= w + 0.5, q <= k/near (1 + 2^-22).
    const double M = std::ldexp(((double)w + 1.5 + (double)k / (double)near_) * (1.0 + 1.0 / 1024.0), -20);
    f->half_m = M < 0.5 ? (float)(0.5 - M) : 0.0f;  // rounding of 0.5 - M: below 2^-25, inside the slack
    f->band = 1;
    f->bulk = (w % 4 == 0) && aligned(color, 16) && aligned(depth, 16) && aligned(out, 16) && aligned(mask, 4);
    f->halo = 1;  // the paper's kernel (h = 3, farthest column first) unless a handle says otherwise
    f->nearest = 0;
    f->zt_out = nullptr;
    return YORO_OK;
}

// The handle's Patcher kernel shape on a frame description.
void apply_options(const yoro_ctx* c, FrameArgs* f)
{
    f->halo = c->halo;
    f->nearest = c->nearest;
}

yoro_status on_device(const yoro_ctx* c)
{
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) return YORO_ECUDA;
    return dev == c->device ? YORO_OK : YORO_EINVAL;
}

yoro_status run_unfused(yoro_ctx* c, const FrameArgs& f, cudaStream_t s)
{
    if (!c->d_zbuf) {
        if (cudaMalloc(&c->d_zbuf, (size_t)c->w * c->h * sizeof(unsigned long long)) != cudaSuccess) {
            c->d_zbuf = nullptr;
            cudaGetLastError();
            return YORO_ENOMEM;
        }
    }
    return yoro::unfused_launch(f, c->d_zbuf, s) == cudaSuccess ? YORO_OK : YORO_ECUDA;
}

// The handle's frames through the row-downsampled intermediate buffer.
// banded: one band kernel when a band's window and cell keys fit (the handle's fused
// calls); otherwise, and for the unfused call, the separate kernels.
yoro_status run_imb(yoro_ctx* c, const FrameArgs& f, cudaStream_t s, bool banded)
{
    if (banded && c->fused_ok && yoro::imb_band_max(c->lim, c->w, c->halo, c->imb_div) >= 1)
        return yoro::imb_band_launch(f, c->imb_div, c->imb_interp, c->lim, s) == cudaSuccess ? YORO_OK : YORO_ECUDA;
    if (!c->d_imb) {
        if (cudaMalloc(&c->d_imb, yoro::imb_scratch_bytes(c->w, c->h, c->imb_div)) != cudaSuccess) {
            c->d_imb = nullptr;
            cudaGetLastError();
            return YORO_ENOMEM;
        }
    }
    const yoro::ImbArgs a = yoro::imb_args(c->d_imb, c->w, c->h, c->imb_div, c->imb_interp);
    return yoro::imb_launch(f, a, c->lim, c->fused_ok, s) == cudaSuccess ? YORO_OK : YORO_ECUDA;
}

bool uses_imb(const yoro_ctx* c) { return c->imb_div > 1 || c->imb_interp; }

// The handle's frames with a general second-eye pose.
yoro_status run_pose(yoro_ctx* c, const FrameArgs& f, cudaStream_t s)
{
    if (!c->d_pose) {
        if (cudaMalloc(&c->d_pose, yoro::pose_scratch_bytes(c->w, c->h)) != cudaSuccess) {
            c->d_pose = nullptr;
            cudaGetLastError();
            return YORO_ENOMEM;
        }
    }
    yoro::PoseArgs p = c->pose_args;
    yoro::pose_bind_scratch(&p, c->d_pose, c->w, c->h);
    return yoro::pose_launch(f, p, c->lim, c->fused_ok, s) == cudaSuccess ? YORO_OK : YORO_ECUDA;
}

yoro_status run_frame(yoro_ctx* c, FrameArgs f, cudaStream_t s)
{
    if (c->pose) return run_pose(c, f, s);
    if (uses_imb(c)) return run_imb(c, f, s, true);
    if (!c->fused_ok) return run_unfused(c, f, s);
    f.band = c->shape.band;
    return yoro::fused_launch(f, c->lim, c->shape.two_per_sm, s) == cudaSuccess ? YORO_OK : YORO_ECUDA;
}

}  // namespace

namespace yoro {
bool camera_valid(int w, int h, float fx, float fy, float cx, float cy, float ipd, float near_, float far_)
{
    return camera_ok(w, h, fx, fy, cx, cy, ipd, near_, far_);
}
int checked_frame(int w, int h, float k, float near_, float far_, const void* color, const float* depth, void* out,
                  unsigned char* mask, FrameArgs* f)
{
    return (int)make_frame(w, h, k, near_, far_, color, depth, out, mask, f);
}
void set_last_create_error(int st) { g_last_create = (yoro_status)st; }
}  // namespace yoro

extern "C" {

yoro_handle yoro_create(int w, int h, float fx, float fy, float cx, float cy, float ipd, float near_, float far_)
{
    return yoro_create_ex(w, h, fx, fy, cx, cy, ipd, near_, far_, nullptr);
}

yoro_handle yoro_create_ex(int w, int h, float fx, float fy, float cx, float cy, float ipd, float near_,
                           float far_, const yoro_options* opt)
{
    const int kernel_rows = opt ? opt->kernel_rows : 3;
    const int nearest = opt ? opt->nearest_first : 0;
    if (!camera_ok(w, h, fx, fy, cx, cy, ipd, near_, far_) || kernel_rows < 1 || kernel_rows > 15 ||
        (kernel_rows & 1) == 0 || (nearest != 0 && nearest != 1)) {
        g_last_create = YORO_EINVAL;
        return nullptr;
    }
    yoro_ctx* c = new (std::nothrow) yoro_ctx();
    if (!c) {
        g_last_create = YORO_ENOMEM;
        return nullptr;
    }
    c->w = w;
    c->h = h;
    c->fx = fx;
    c->fy = fy;
    c->cx = cx;
    c->cy = cy;
    c->ipd = ipd;
    c->near_ = near_;
    c->far_ = far_;
    c->k = fx * ipd;  // one binary32 rounding, shared by every pixel
    if (cudaGetDevice(&c->device) != cudaSuccess || yoro::fused_configure(c->device, &c->lim) != cudaSuccess) {
        cudaGetLastError();
        delete c;
        g_last_create = YORO_ECUDA;
        return nullptr;
    }
    c->halo = (kernel_rows - 1) / 2;
    c->nearest = nearest;
    c->imb_div = 1;
    c->imb_interp = 0;
    c->fused_ok = w <= c->lim.max_width &&
                  yoro::fused_smem_bytes(yoro::fused_wpad(w), 1, c->halo) <= (size_t)c->lim.smem_per_block;
    c->shape = yoro::fused_shape(c->lim, w, h, c->halo);
    g_last_create = YORO_OK;
    return c;
}

yoro_handle yoro_create_imb(int w, int h, float fx, float fy, float cx, float cy, float ipd, float near_, float far_,
                            const yoro_options* opt, int imbuffer_div, int interpolate)
{
    if ((imbuffer_div != 1 && imbuffer_div != 2 && imbuffer_div != 4 && imbuffer_div != 8 && imbuffer_div != 16) ||
        (interpolate != 0 && interpolate != 1)) {
        g_last_create = YORO_EINVAL;
        return nullptr;
    }
    yoro_ctx* c = yoro_create_ex(w, h, fx, fy, cx, cy, ipd, near_, far_, opt);
    if (!c) return nullptr;
    c->imb_div = imbuffer_div;
    c->imb_interp = interpolate;
    return c;
}

yoro_handle yoro_create_pose(int w, int h, float fx, float fy, float cx, float cy, const float* rotation,
                             const float* position, float near_, float far_, const yoro_options* opt)
{
    if (!rotation || !position) {
        g_last_create = YORO_EINVAL;
        return nullptr;
    }
    for (int i = 0; i < 9; ++i)
        if (!std::isfinite(rotation[i])) {
            g_last_create = YORO_EINVAL;
            return nullptr;
        }
    for (int i = 0; i < 3; ++i)
        if (!std::isfinite(position[i])) {
            g_last_create = YORO_EINVAL;
            return nullptr;
        }
    if (!(fy > 0.0f)) {
        g_last_create = YORO_EINVAL;
        return nullptr;
    }
    yoro_ctx* c = yoro_create_ex(w, h, fx, fy, cx, cy, 0.0f, near_, far_, opt);
    if (!c) return nullptr;
    c->pose = true;
    c->pose_args.fx = fx;
    c->pose_args.fy = fy;
    c->pose_args.cx = cx;
    c->pose_args.cy = cy;
    for (int i = 0; i < 9; ++i) c->pose_args.rot[i] = rotation[i];
    for (int i = 0; i < 3; ++i) c->pose_args.c[i] = position[i];
    c->pose_args.zbuf = nullptr;
    c->pose_args.zt = nullptr;
    return c;
}

yoro_status yoro_last_create_error(void) { return g_last_create; }

void yoro_destroy(yoro_handle c)
{
    if (!c) return;
    if (c->d_zbuf) cudaFree(c->d_zbuf);
    if (c->d_stage) cudaFree(c->d_stage);
    if (c->d_imb) cudaFree(c->d_imb);
    if (c->d_pose) cudaFree(c->d_pose);
    delete c;
}

yoro_status yoro_synthesize(yoro_handle c, const void* color, const float* depth, void* out_color,
                            unsigned char* out_mask, void* stream)
{
    if (!c) return YORO_EINVAL;
    if ((size_t)c->w * c->h == 0) return YORO_OK;
    yoro_status st = on_device(c);
    if (st != YORO_OK) return st;
    FrameArgs f;
    st = make_frame(c->w, c->h, c->k, c->near_, c->far_, color, depth, out_color, out_mask, &f);
    if (st != YORO_OK) return st;
    apply_options(c, &f);
    return run_frame(c, f, (cudaStream_t)stream);
}

yoro_status yoro_synthesize_zt(yoro_handle c, const void* color, const float* depth, void* out_color,
                               unsigned char* out_mask, float* out_zt, void* stream)
{
    if (!c) return YORO_EINVAL;
    if ((size_t)c->w * c->h == 0) return YORO_OK;
    yoro_status st = on_device(c);
    if (st != YORO_OK) return st;
    // the fused kernel with the paper's Patcher only
    if (c->pose || uses_imb(c) || !c->fused_ok || c->halo != 1 || c->nearest) return YORO_EINVAL;
    FrameArgs f;
    st = make_frame(c->w, c->h, c->k, c->near_, c->far_, color, depth, out_color, out_mask, &f);
    if (st != YORO_OK) return st;
    const size_t n = (size_t)c->w * c->h;
    if (!out_zt) return YORO_EINVAL;
    if ((uintptr_t)out_zt & 3u) return YORO_EALIGN;
    if (overlaps(out_zt, 4 * n, color, 4 * n) || overlaps(out_zt, 4 * n, depth, 4 * n) ||
        overlaps(out_zt, 4 * n, out_color, 4 * n) || overlaps(out_zt, 4 * n, out_mask, n))
        return YORO_EINVAL;
    f.zt_out = out_zt;
    f.band = c->shape.band;
    return yoro::fused_launch(f, c->lim, c->shape.two_per_sm, (cudaStream_t)stream) == cudaSuccess ? YORO_OK
                                                                                                 : YORO_ECUDA;
}

yoro_status yoro_synthesize_unfused(yoro_handle c, const void* color, const float* depth, void* out_color,
                                    unsigned char* out_mask, void* stream)
{
    if (!c) return YORO_EINVAL;
    if ((size_t)c->w * c->h == 0) return YORO_OK;
    yoro_status st = on_device(c);
    if (st != YORO_OK) return st;
    FrameArgs f;
    st = make_frame(c->w, c->h, c->k, c->near_, c->far_, color, depth, out_color, out_mask, &f);
    if (st != YORO_OK) return st;
    apply_options(c, &f);
    if (c->pose) return run_pose(c, f, (cudaStream_t)stream);
    if (uses_imb(c)) return run_imb(c, f, (cudaStream_t)stream, false);
    return run_unfused(c, f, (cudaStream_t)stream);
}

yoro_status yoro_synthesize_mapped(yoro_handle c, const void* hcolor, const float* hdepth, void* hout,
                                   unsigned char* hmask, void* stream)
{
    if (!c) return YORO_EINVAL;
    if ((size_t)c->w * c->h == 0) return YORO_OK;
    if (!hcolor || !hdepth || !hout || !hmask) return YORO_EINVAL;
    yoro_status st = on_device(c);
    if (st != YORO_OK) return st;
    // Every buffer must be page-locked host memory mapped into the device address space:
    // the kernels then load and store it directly, and nothing else is accepted.
    const void* hp[4] = {hcolor, hdepth, hout, hmask};
    void* dp[4];
    for (int i = 0; i < 4; ++i) {
        cudaPointerAttributes a;
        if (cudaPointerGetAttributes(&a, hp[i]) != cudaSuccess || a.type != cudaMemoryTypeHost ||
            !a.devicePointer) {
            cudaGetLastError();
            return YORO_EINVAL;
        }
        dp[i] = a.devicePointer;
    }
    FrameArgs f;
    st = make_frame(c->w, c->h, c->k, c->near_, c->far_, dp[0], (const float*)dp[1], dp[2], (unsigned char*)dp[3],
                    &f);
    if (st != YORO_OK) return st;
    f.bulk = 0;  // no L2 bulk prefetch of host memory
    apply_options(c, &f);
    return run_frame(c, f, (cudaStream_t)stream);
}

yoro_status yoro_synthesize_host(yoro_handle c, const void* hcolor, const float* hdepth, void* hout,
                                 unsigned char* hmask, void* stream)
{
    if (!c) return YORO_EINVAL;
    const size_t n = (size_t)c->w * c->h;
    if (n == 0) return YORO_OK;
    if (!hcolor || !hdepth || !hout || !hmask) return YORO_EINVAL;
    yoro_status st = on_device(c);
    if (st != YORO_OK) return st;
    const size_t seg = (4 * n + 255) & ~(size_t)255;
    if (!c->d_stage) {
        if (cudaMalloc(&c->d_stage, 3 * seg + n) != cudaSuccess) {
            c->d_stage = nullptr;
            cudaGetLastError();
            return YORO_ENOMEM;
        }
    }
    unsigned char* dc = c->d_stage;
    float* dd = (float*)(c->d_stage + seg);
    unsigned char* dout = c->d_stage + 2 * seg;
    unsigned char* dmask = c->d_stage + 3 * seg;
    cudaStream_t s = (cudaStream_t)stream;
    if (cudaMemcpyAsync(dc, hcolor, 4 * n, cudaMemcpyHostToDevice, s) != cudaSuccess ||
        cudaMemcpyAsync(dd, hdepth, 4 * n, cudaMemcpyHostToDevice, s) != cudaSuccess)
        return YORO_ECUDA;
    FrameArgs f;
    st = make_frame(c->w, c->h, c->k, c->near_, c->far_, dc, dd, dout, dmask, &f);
    if (st != YORO_OK) return st;
    apply_options(c, &f);
    st = run_frame(c, f, s);
    if (st != YORO_OK) return st;
    if (cudaMemcpyAsync(hout, dout, 4 * n, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaMemcpyAsync(hmask, dmask, n, cudaMemcpyDeviceToHost, s) != cudaSuccess)
        return YORO_ECUDA;
    return YORO_OK;
}

}  // extern "C"

namespace {

// Band heights chosen by yoro_tune_batch, per (device, widest frame width of a launch).
std::mutex g_tune_mutex;
std::map<std::pair<int, int>, int> g_tuned_band;

// Rows per work item of a batch launch whose widest frame is wmax: the tuned height if
// one was measured for this device and width, else the tallest that fits shared memory.
int batch_band(int dev, const FusedLimits& lim, int wmax)
{
    const int bmax = yoro::fused_max_band(lim, wmax);
    std::lock_guard<std::mutex> lock(g_tune_mutex);
    const auto it = g_tuned_band.find({dev, wmax});
    if (it != g_tuned_band.end() && it->second >= 1 && it->second <= bmax) return it->second;
    return bmax;
}

// Checks every frame of a batch (before anything is launched); returns the widest width.
yoro_status batch_validate(int n, const yoro_frame* frames, const FusedLimits& lim, int* wmax_out)
{
    int wmax = 0;
    for (int i = 0; i < n; ++i) {
        const yoro_frame& fr = frames[i];
        if (!camera_ok(fr.w, fr.h, fr.fx, fr.fy, fr.cx, fr.cy, fr.ipd, fr.near_, fr.far_)) return YORO_EINVAL;
        if (fr.w > lim.max_width) return YORO_ETOOBIG;
        if ((size_t)fr.w * fr.h == 0) continue;
        FrameArgs f;
        const yoro_status st = make_frame(fr.w, fr.h, fr.fx * fr.ipd, fr.near_, fr.far_, fr.color, fr.depth,
                                          fr.out_color, fr.out_hole_mask, &f);
        if (st != YORO_OK) return st;
        wmax = std::max(wmax, fr.w);
    }
    if (wmax_out) *wmax_out = wmax;
    return YORO_OK;
}

// Launches validated frames, up to kMaxBatch per launch.  band_override > 0 sets the rows
// per work item of every launch (it must fit the widest frame); 0 takes batch_band().
yoro_status batch_launch(int n, const yoro_frame* frames, int dev, const FusedLimits& lim, int band_override,
                         cudaStream_t stream, float* const* zt = nullptr)
{
    yoro::BatchArgs* a = new (std::nothrow) yoro::BatchArgs;
    if (!a) return YORO_ENOMEM;
    yoro_status result = YORO_OK;
    int i = 0;
    while (i < n && result == YORO_OK) {
        int i1 = i, wmax = 0, cnt = 0;
        for (; i1 < n && cnt < yoro::kMaxBatch; ++i1) {
            if ((size_t)frames[i1].w * frames[i1].h == 0) continue;
            if (frames[i1].w > wmax) wmax = frames[i1].w;
            ++cnt;
        }
        const int band = band_override > 0 ? band_override : batch_band(dev, lim, wmax);
        // the launch's shared memory holds `band` rows of the widest frame; a narrower
        // frame's window uses its own row stride, so its bands take as many rows as fit
        const size_t smem = yoro::fused_smem_bytes(yoro::fused_wpad(wmax), band, 1);
        a->n = 0;
        a->total_items = 0;
        a->max_band = band;
        for (; i < i1; ++i) {
            const yoro_frame& fr = frames[i];
            if ((size_t)fr.w * fr.h == 0) continue;
            FrameArgs f;
            make_frame(fr.w, fr.h, fr.fx * fr.ipd, fr.near_, fr.far_, fr.color, fr.depth, fr.out_color,
                       fr.out_hole_mask, &f);
            int fb = band;
            while (fb < fr.h && yoro::fused_smem_bytes(yoro::fused_wpad(fr.w), fb + 1, 1) <= smem) ++fb;
            f.band = fb;
            f.zt_out = zt ? zt[i] : nullptr;
            a->item_start[a->n] = a->total_items;
            a->f[a->n++] = f;
            a->total_items += (f.h + f.band - 1) / f.band;
        }
        a->item_start[a->n] = a->total_items;
        if (a->n > 0 && yoro::fused_launch_batch(*a, wmax, lim, stream, zt != nullptr) != cudaSuccess)
            result = YORO_ECUDA;
    }
    delete a;
    return result;
}

}  // namespace

namespace yoro {
int synthesize_batch_zt(int n, const yoro_frame* frames, float* const* zt, cudaStream_t stream)
{
    if (n < 0 || (n > 0 && !frames)) return YORO_EINVAL;
    if (n > 4096) return YORO_ETOOBIG;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return YORO_ECUDA;
    FusedLimits lim;
    if (yoro::fused_configure(dev, &lim) != cudaSuccess) return YORO_ECUDA;
    const yoro_status st = batch_validate(n, frames, lim, nullptr);
    if (st != YORO_OK) return st;
    return batch_launch(n, frames, dev, lim, 0, stream, zt);
}
}  // namespace yoro

extern "C" {

yoro_status yoro_synthesize_batch(int n, const yoro_frame* frames, void* stream)
{
    if (n < 0 || (n > 0 && !frames)) return YORO_EINVAL;
    if (n > 4096) return YORO_ETOOBIG;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return YORO_ECUDA;
    FusedLimits lim;
    if (yoro::fused_configure(dev, &lim) != cudaSuccess) return YORO_ECUDA;
    const yoro_status st = batch_validate(n, frames, lim, nullptr);  // before launching anything
    if (st != YORO_OK) return st;
    return batch_launch(n, frames, dev, lim, 0, (cudaStream_t)stream);
}

yoro_status yoro_tune_batch(int n, const yoro_frame* frames, int reps, void* stream, int* out_band)
{
    if (n <= 0 || !frames || reps < 1 || reps > 1000) return YORO_EINVAL;
    if (n > 4096) return YORO_ETOOBIG;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return YORO_ECUDA;
    FusedLimits lim;
    if (yoro::fused_configure(dev, &lim) != cudaSuccess) return YORO_ECUDA;
    int wmax = 0;
    yoro_status st = batch_validate(n, frames, lim, &wmax);
    if (st != YORO_OK) return st;
    if (wmax == 0) return YORO_EINVAL;  // nothing to time
    // Candidates: the tallest band, a few just below it, and fractions of it (the
    // shorter ones fit two CTAs per SM and run the 512-thread shape).
    const int bmax = yoro::fused_max_band(lim, wmax);
    std::vector<int> cand = {bmax, bmax - 1, bmax - 2, (3 * bmax + 3) / 4, (bmax + 1) / 2, (bmax + 2) / 3,
                             (bmax + 3) / 4};
    std::sort(cand.begin(), cand.end());
    cand.erase(std::unique(cand.begin(), cand.end()), cand.end());
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        if (e0) cudaEventDestroy(e0);
        cudaGetLastError();
        return YORO_ECUDA;
    }
    const cudaStream_t s = (cudaStream_t)stream;
    int best = bmax;
    float best_ms = 0.0f;
    bool have = false;
    for (const int band : cand) {
        if (band < 1 || band > bmax) continue;
        st = batch_launch(n, frames, dev, lim, band, s);  // warm-up
        for (int r = 0; r < reps && st == YORO_OK; ++r) {
            if (r == 0 && cudaEventRecord(e0, s) != cudaSuccess) st = YORO_ECUDA;
            if (st == YORO_OK) st = batch_launch(n, frames, dev, lim, band, s);
        }
        float ms = 0.0f;
        if (st == YORO_OK && (cudaEventRecord(e1, s) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
                              cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess))
            st = YORO_ECUDA;
        if (st != YORO_OK) break;
        if (!have || ms < best_ms) {
            best = band;
            best_ms = ms;
            have = true;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st != YORO_OK) {
        cudaGetLastError();
        return st;
    }
    {
        std::lock_guard<std::mutex> lock(g_tune_mutex);
        g_tuned_band[{dev, wmax}] = best;
    }
    if (out_band) *out_band = best;
    return YORO_OK;
}

int yoro_batch_band(int w)
{
    int dev = 0;
    FusedLimits lim;
    if (w < 1 || cudaGetDevice(&dev) != cudaSuccess || yoro::fused_configure(dev, &lim) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    if (w > lim.max_width) return 0;
    return batch_band(dev, lim, w);
}

void yoro_reset_tuning(void)
{
    std::lock_guard<std::mutex> lock(g_tune_mutex);
    g_tuned_band.clear();
}

yoro_status yoro_stream_status(yoro_handle c, void* stream)
{
    (void)c;
    if (cudaStreamSynchronize((cudaStream_t)stream) != cudaSuccess) {
        cudaGetLastError();
        return YORO_ECUDA;
    }
    if (cudaPeekAtLastError() != cudaSuccess) return YORO_ECUDA;
    // both words are read (and cleared) whichever is set
    const unsigned bad =
        yoro::fused_status_take() | yoro::unfused_status_take() | yoro::imb_status_take() | yoro::pose_status_take();
    return bad ? YORO_EDEVICE : YORO_OK;
}

int yoro_debug_bounds_enabled(void) { return yoro::debug_bounds_built() ? 1 : 0; }

yoro_status yoro_debug_selftest(void* stream)
{
    return yoro::debug_selftest_launch((cudaStream_t)stream) == cudaSuccess ? YORO_OK : YORO_ECUDA;
}

int yoro_max_fused_width(void)
{
    int dev = 0;
    FusedLimits lim;
    if (cudaGetDevice(&dev) != cudaSuccess || yoro::fused_configure(dev, &lim) != cudaSuccess) return 0;
    return lim.max_width;
}

const char* yoro_status_string(yoro_status s)
{
    switch (s) {
        case YORO_OK: return "ok";
        case YORO_EINVAL: return "invalid argument";
        case YORO_EALIGN: return "pointer not 4-byte aligned";
        case YORO_ENOMEM: return "allocation failed";
        case YORO_ECUDA: return "CUDA error";
        case YORO_EDEVICE: return "kernel reported an error";
        case YORO_ETOOBIG: return "frame exceeds a limit of this entry point";
        case YORO_ETIMEOUT: return "a wait ran out of time";
        case YORO_ECANCELED: return "cancelled before it ran";
    }
    return "unknown status";
}

}  // extern "C"
