// Serving loop: admitted streams with resident frame slots, continuous batching by a
// scheduler thread.  Contract in include/yoro_server.h.
//
// The scheduler keeps up to four batches in flight on its own CUDA stream: it launches
// whatever is pending as one batched synthesis, and while that runs, gathers the frames
// submitted meanwhile into the next launch; it then waits (a blocking-sync CUDA event, so
// the thread sleeps) for the older batch and reports its frames complete.  Frames of
// streams admitted with learned inpainting also get their warped depth from the batch,
// and then, on a second CUDA stream ordered after the synthesis by an event, the server's
// inpainter repaints their holes; a host function enqueued after them reports those
// frames, so a batch retires, and the scheduler moves on, as soon as its synthesis is
// done.  Without an inpainter (or for a frame larger than it takes) learned frames keep
// the paper's fill and complete with the batch.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstdint>
#include <deque>
#include <mutex>
#include <new>
#include <thread>
#include <vector>

#include "yoro.h"
#include "yoro_internal.h"
#include "yoro_server.h"
#include "yoro_unet.h"

namespace yoro {
// api.cu: yoro_synthesize_batch, where frame i with zt[i] set also writes its warped depth
// there; returns a yoro_status.
int synthesize_batch_zt(int n, const yoro_frame* frames, float* const* zt, cudaStream_t stream);
}  // namespace yoro

namespace {

long long now_ns()
{
    return std::chrono::duration_cast<std::chrono::nanoseconds>(std::chrono::steady_clock::now().time_since_epoch())
        .count();
}

size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

struct Slot {
    void* color;
    float* depth;
    void* out;
    unsigned char* mask;
    float* zt;  // warped depth (streams with learned inpainting), else null
    bool in_flight;
};

struct Stream {
    bool live = false;
    int w = 0, h = 0;
    float fx = 0, fy = 0, cx = 0, cy = 0, ipd = 0, near_ = 0, far_ = 0;
    size_t bytes = 0;
    unsigned char* block = nullptr;
    std::vector<Slot> slots;
    int pending = 0;  // submitted, not completed
    bool learned = false;
};

struct Request {
    int stream, slot;
    unsigned long long tag;
    long long submit_ns;
    int inpainted;
    int learned;  // the frame's stream repaints holes with the inpainter
};

// A feeding job (yoro_server_feed): source frames copied into the stream's free slots
// and submitted by the server's feeder thread.
struct FeedJob {
    int stream;
    std::vector<const void*> colors;
    std::vector<const float*> depths;
    long long remaining;
    long long next;          // index of the next source frame (cyclic)
    double period_ns;        // 0: as fast as slots free up
    long long due_ns;        // when the next frame may go (paced jobs)
    unsigned long long tag;  // tag of the next frame
};

struct Batch {
    std::vector<Request> req;
    cudaEvent_t synth = nullptr;  // the batched synthesis is done (plain frames complete here)
    cudaEvent_t done = nullptr;   // the learned frames' inpainting is done too
    long long launch_ns = 0;
    yoro_status status = YORO_OK;
    bool any_learned = false;
    int frames = 0;  // frames launched in this batch (learned ones included)
};

struct LearnedDone;  // learned frames of one batch, reported by a host function on the inpainting stream

constexpr int kMaxSlots = 64;
constexpr int kInFlight = 4;

}  // namespace

struct yoro_server_ctx {
    int device = 0;
    size_t budget = 0, used = 0;
    int max_batch = 0;
    cudaStream_t cs = nullptr;  // synthesis
    cudaStream_t ci = nullptr;  // learned inpainting, after each batch's synthesis (its own queue,
                                // so the next batch's synthesis does not wait behind it)
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<Request> pending;
    std::deque<yoro_completion> done;
    std::vector<Stream> streams;
    long long outstanding = 0;  // submitted and not completed
    bool stop = false;
    bool paused = false;
    yoro_unet inpainter = nullptr;
    Batch ring[kInFlight];
    std::thread worker;
    // feeder
    std::vector<FeedJob> jobs;
    std::thread feeder;
    bool feeder_started = false;
    cudaStream_t fs = nullptr;

    void run();
    void feed_loop();
    void complete(Batch& b, long long t_done, int which);
    void report(const std::vector<Request>& reqs, long long launch_ns, int batch_frames, yoro_status status,
                long long t_done);
};

namespace {
struct LearnedDone {
    yoro_server_ctx* server;
    std::vector<Request> req;
    long long launch_ns;
    int batch_frames;
};

// Runs on the CUDA runtime's thread once the inpainting enqueued before it is done; it
// touches host state only (no CUDA call is allowed here).
void CUDART_CB learned_done(void* p)
{
    LearnedDone* d = static_cast<LearnedDone*>(p);
    d->server->report(d->req, d->launch_ns, d->batch_frames, YORO_OK, now_ns());
    delete d;
}
}  // namespace

void yoro_server_ctx::report(const std::vector<Request>& reqs, long long launch_ns, int batch_frames,
                             yoro_status status, long long t_done)
{
    {
        std::lock_guard<std::mutex> lk(mu);
        for (const Request& r : reqs) {
            yoro_completion c;
            c.stream = r.stream;
            c.slot = r.slot;
            c.tag = r.tag;
            c.submit_ns = r.submit_ns;
            c.launch_ns = launch_ns;
            c.done_ns = t_done;
            c.batch_frames = batch_frames;
            c.status = status;
            c.inpainted = status == YORO_OK ? r.inpainted : 0;
            done.push_back(c);
            Stream& st = streams[r.stream];
            st.slots[r.slot].in_flight = false;
            --st.pending;
            --outstanding;
        }
    }
    cv_done.notify_all();
}

// which: 0 the plain frames of the batch, 1 the learned ones, 2 all; the batch's request
// list is cleared once its last frames are reported.
void yoro_server_ctx::complete(Batch& b, long long t_done, int which)
{
    {
        std::lock_guard<std::mutex> lk(mu);
        for (const Request& r : b.req) {
            const bool learned_frame = r.learned != 0;
            if ((which == 0 && learned_frame) || (which == 1 && !learned_frame)) continue;
            yoro_completion c;
            c.stream = r.stream;
            c.slot = r.slot;
            c.tag = r.tag;
            c.submit_ns = r.submit_ns;
            c.launch_ns = b.launch_ns;
            c.done_ns = t_done;
            c.batch_frames = b.frames;
            c.status = b.status;
            c.inpainted = b.status == YORO_OK ? r.inpainted : 0;
            done.push_back(c);
            Stream& st = streams[r.stream];
            st.slots[r.slot].in_flight = false;
            --st.pending;
            --outstanding;
        }
        if (which != 0) b.req.clear();
    }
    cv_done.notify_all();
}

void yoro_server_ctx::run()
{
    cudaSetDevice(device);
    std::vector<yoro_frame> frames;
    std::vector<float*> zts;
    yoro_unet net = nullptr;
    int head = 0, count = 0;  // ring of batches in flight: oldest at head
    for (;;) {
        // Launch a new batch when one can be in flight and work is pending; otherwise
        // wait for the oldest batch or for work.
        bool launched = false;
        if (count < kInFlight) {
            Batch& b = ring[(head + count) % kInFlight];
            {
                std::unique_lock<std::mutex> lk(mu);
                if (count == 0) cv_work.wait(lk, [&] { return stop || (!paused && !pending.empty()); });
                if (pending.empty() && count == 0 && stop) break;
                frames.clear();
                zts.clear();
                net = inpainter;
                while (!paused && !pending.empty() && (int)b.req.size() < max_batch) {
                    const Request r = pending.front();
                    pending.pop_front();
                    const Stream& st = streams[r.stream];
                    const Slot& sl = st.slots[r.slot];
                    yoro_frame f;
                    f.w = st.w;
                    f.h = st.h;
                    f.fx = st.fx;
                    f.fy = st.fy;
                    f.cx = st.cx;
                    f.cy = st.cy;
                    f.ipd = st.ipd;
                    f.near_ = st.near_;
                    f.far_ = st.far_;
                    f.color = sl.color;
                    f.depth = sl.depth;
                    f.out_color = sl.out;
                    f.out_hole_mask = sl.mask;
                    frames.push_back(f);
                    zts.push_back(st.learned ? sl.zt : nullptr);
                    b.req.push_back(r);
                    b.req.back().learned = st.learned ? 1 : 0;
                }
            }
            if (!b.req.empty()) {
                b.launch_ns = now_ns();
                bool any_learned = false;
                for (float* z : zts) any_learned = any_learned || z != nullptr;
                b.status = (yoro_status)yoro::synthesize_batch_zt((int)frames.size(), frames.data(),
                                                                  any_learned ? zts.data() : nullptr, cs);
                b.any_learned = any_learned;
                b.frames = (int)b.req.size();
                if (b.status == YORO_OK && cudaEventRecord(b.synth, cs) != cudaSuccess) b.status = YORO_ECUDA;
                // learned inpainting of those frames on the inpainting stream, once the
                // synthesis is done
                cudaStream_t done_on = cs;
                if (b.status == YORO_OK && any_learned && net) {
                    if (cudaStreamWaitEvent(ci, b.synth, 0) != cudaSuccess) b.status = YORO_ECUDA;
                    done_on = ci;
                }
                // all of them in one call: their hole cells share the network's passes
                std::vector<yoro_unet_frame> lf;
                std::vector<size_t> li;
                for (size_t i = 0; i < b.req.size(); ++i) {
                    b.req[i].inpainted = 0;
                    if (b.status != YORO_OK || !zts[i] || !net) continue;
                    const yoro_frame& f = frames[i];
                    lf.push_back(yoro_unet_frame{f.w, f.h, f.near_, f.out_color, f.out_hole_mask, zts[i], f.depth});
                    li.push_back(i);
                }
                if (!lf.empty()) {
                    if (yoro_unet_inpaint_batch(net, (int)lf.size(), lf.data(), ci) == YORO_OK) {
                        for (size_t i : li) b.req[i].inpainted = 1;
                    } else {  // a frame the inpainter does not take: the others one by one
                        for (size_t k = 0; k < lf.size(); ++k) {
                            const yoro_unet_frame& u = lf[k];
                            b.req[li[k]].inpainted = yoro_unet_inpaint(net, u.w, u.h, u.near_, u.rgba, u.mask, u.zt,
                                                                       u.src_depth, ci) == YORO_OK;
                        }
                    }
                }
                // The learned frames are reported by a host function after their inpainting, so
                // that the batch retires (and the scheduler moves on) when the synthesis is done.
                if (b.status == YORO_OK && done_on == ci) {
                    LearnedDone* ld = new (std::nothrow) LearnedDone();
                    if (ld) {
                        ld->server = this;
                        ld->launch_ns = b.launch_ns;
                        ld->batch_frames = (int)b.req.size();
                        std::vector<Request> plain;
                        for (const Request& r : b.req) (r.learned ? ld->req : plain).push_back(r);
                        if (cudaLaunchHostFunc(ci, learned_done, ld) == cudaSuccess) {
                            b.req.swap(plain);
                            b.any_learned = false;
                            done_on = cs;
                        } else {
                            cudaGetLastError();
                            delete ld;
                        }
                    }
                }
                if (b.status == YORO_OK && cudaEventRecord(b.done, done_on) != cudaSuccess) b.status = YORO_ECUDA;
                ++count;
                launched = true;
            }
        }
        if (count == 0) continue;
        if (launched && count < kInFlight) continue;  // gather the next batch while this one runs
        Batch& old = ring[head];
        bool plain_reported = false;
        if (old.any_learned && old.status == YORO_OK) {  // plain frames leave when the synthesis is done
            if (cudaEventSynchronize(old.synth) != cudaSuccess) old.status = YORO_ECUDA;
            if (old.status == YORO_OK) {
                complete(old, now_ns(), 0);
                plain_reported = true;
            }
        }
        if (old.status == YORO_OK && cudaEventSynchronize(old.done) != cudaSuccess) old.status = YORO_ECUDA;
        if (old.status != YORO_OK) cudaGetLastError();
        complete(old, now_ns(), plain_reported ? 1 : 2);
        head = (head + 1) % kInFlight;
        --count;
    }
}

void yoro_server_ctx::feed_loop()
{
    cudaSetDevice(device);
    std::unique_lock<std::mutex> lk(mu);
    for (;;) {
        if (stop) break;
        const long long now = now_ns();
        long long wake = -1;  // earliest due time of a paced job waiting for its time
        bool progressed = false;
        for (size_t j = 0; j < jobs.size(); ++j) {
            FeedJob& jb = jobs[j];
            if (jb.remaining <= 0) continue;
            Stream& st = streams[jb.stream];
            if (!st.live) {
                jb.remaining = 0;
                continue;
            }
            if (jb.period_ns > 0 && now < jb.due_ns) {
                wake = wake < 0 ? jb.due_ns : std::min(wake, jb.due_ns);
                continue;
            }
            int k = -1;
            for (int i = 0; i < (int)st.slots.size(); ++i)
                if (!st.slots[i].in_flight) {
                    k = i;
                    break;
                }
            if (k < 0) continue;  // every slot busy: a completion wakes us
            // Reserve the slot and count the frame as pending before the lock is dropped
            // (leave() then waits for it); take plain values only: admit() or feed() may
            // grow the vectors while the copy runs.
            st.slots[k].in_flight = true;
            ++st.pending;
            ++outstanding;
            void* dst_c = st.slots[k].color;
            float* dst_d = st.slots[k].depth;
            const size_t n = (size_t)st.w * st.h;
            const void* c = jb.colors[jb.next % jb.colors.size()];
            const float* d = jb.depths[jb.next % jb.depths.size()];
            const int sid = jb.stream;
            const unsigned long long tag = jb.tag++;
            ++jb.next;
            --jb.remaining;
            if (jb.period_ns > 0) jb.due_ns += (long long)jb.period_ns;
            lk.unlock();
            const bool ok = cudaMemcpyAsync(dst_c, c, 4 * n, cudaMemcpyDeviceToDevice, fs) == cudaSuccess &&
                            cudaMemcpyAsync(dst_d, d, 4 * n, cudaMemcpyDeviceToDevice, fs) == cudaSuccess &&
                            cudaStreamSynchronize(fs) == cudaSuccess;
            lk.lock();
            if (!ok) {
                cudaGetLastError();
                streams[sid].slots[k].in_flight = false;
                --streams[sid].pending;
                --outstanding;
                cv_done.notify_all();
                continue;
            }
            pending.push_back(Request{sid, k, tag, now_ns(), 0, 0});
            cv_work.notify_one();
            progressed = true;
        }
        if (progressed) continue;
        bool any = false;
        for (const FeedJob& jb : jobs) any = any || jb.remaining > 0;
        if (!any) {
            cv_done.wait(lk, [&] {
                if (stop) return true;
                for (const FeedJob& jb : jobs)
                    if (jb.remaining > 0) return true;
                return false;
            });
        } else if (wake >= 0) {
            cv_done.wait_for(lk, std::chrono::nanoseconds(std::max<long long>(wake - now_ns(), 0)));
        } else {
            cv_done.wait_for(lk, std::chrono::milliseconds(5));
        }
    }
}

extern "C" {

yoro_server yoro_server_create(size_t memory_budget_bytes, int max_batch)
{
    if (memory_budget_bytes == 0 || max_batch < 1 || max_batch > 4096) {
        yoro::set_last_create_error(YORO_EINVAL);
        return nullptr;
    }
    yoro_server_ctx* s = new (std::nothrow) yoro_server_ctx();
    if (!s) {
        yoro::set_last_create_error(YORO_ENOMEM);
        return nullptr;
    }
    s->budget = memory_budget_bytes;
    s->max_batch = max_batch;
    // The synthesis stream gets the highest scheduling priority and the inpainting stream
    // the lowest: pending CTAs of a synthesis launch go to SMs ahead of the network's.
    int prio_low = 0, prio_high = 0;
    bool ok = cudaGetDevice(&s->device) == cudaSuccess &&
              cudaDeviceGetStreamPriorityRange(&prio_low, &prio_high) == cudaSuccess &&
              cudaStreamCreateWithPriority(&s->cs, cudaStreamNonBlocking, prio_high) == cudaSuccess &&
              cudaStreamCreateWithPriority(&s->ci, cudaStreamNonBlocking, prio_low) == cudaSuccess;
    for (int i = 0; ok && i < kInFlight; ++i)
        ok = cudaEventCreateWithFlags(&s->ring[i].done, cudaEventBlockingSync | cudaEventDisableTiming) ==
                 cudaSuccess &&
             cudaEventCreateWithFlags(&s->ring[i].synth, cudaEventBlockingSync | cudaEventDisableTiming) ==
                 cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        for (Batch& b : s->ring) {
            if (b.done) cudaEventDestroy(b.done);
            if (b.synth) cudaEventDestroy(b.synth);
        }
        if (s->cs) cudaStreamDestroy(s->cs);
        if (s->ci) cudaStreamDestroy(s->ci);
        delete s;
        yoro::set_last_create_error(YORO_ECUDA);
        return nullptr;
    }
    try {
        s->worker = std::thread([s] { s->run(); });
    } catch (...) {
        for (Batch& b : s->ring) {
            cudaEventDestroy(b.done);
            cudaEventDestroy(b.synth);
        }
        cudaStreamDestroy(s->cs);
        cudaStreamDestroy(s->ci);
        delete s;
        yoro::set_last_create_error(YORO_ENOMEM);
        return nullptr;
    }
    yoro::set_last_create_error(YORO_OK);
    return s;
}

void yoro_server_destroy(yoro_server s)
{
    if (!s) return;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
        for (FeedJob& jb : s->jobs) jb.remaining = 0;
    }
    s->cv_work.notify_all();
    s->cv_done.notify_all();
    if (s->feeder.joinable()) s->feeder.join();
    if (s->fs) cudaStreamDestroy(s->fs);
    if (s->worker.joinable()) s->worker.join();
    cudaStreamSynchronize(s->cs);
    cudaStreamSynchronize(s->ci);
    for (Stream& st : s->streams)
        if (st.block) cudaFree(st.block);
    for (Batch& b : s->ring) {
        cudaEventDestroy(b.done);
        cudaEventDestroy(b.synth);
    }
    cudaStreamDestroy(s->cs);
    cudaStreamDestroy(s->ci);
    delete s;
}

int yoro_server_admit(yoro_server s, int w, int h, float fx, float fy, float cx, float cy, float ipd, float near_,
                      float far_, int slots)
{
    return yoro_server_admit_ex(s, w, h, fx, fy, cx, cy, ipd, near_, far_, slots, 0);
}

int yoro_server_admit_ex(yoro_server s, int w, int h, float fx, float fy, float cx, float cy, float ipd,
                         float near_, float far_, int slots, int learned)
{
    if (learned != 0 && learned != 1) return -YORO_EINVAL;
    if (!s || slots < 1 || slots > kMaxSlots || !yoro::camera_valid(w, h, fx, fy, cx, cy, ipd, near_, far_) ||
        (size_t)w * (size_t)h == 0)
        return -YORO_EINVAL;
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev != s->device) {
        cudaGetLastError();
        return -YORO_EINVAL;
    }
    if (w > yoro_max_fused_width()) return -YORO_ETOOBIG;
    const size_t n = (size_t)w * (size_t)h;
    const size_t per_slot = (learned ? 4 : 3) * align256(4 * n) + align256(n);
    const size_t bytes = per_slot * (size_t)slots;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        if (s->used + bytes > s->budget) return -YORO_ENOMEM;
        s->used += bytes;  // reserved while the allocation runs
    }
    unsigned char* block = nullptr;
    if (cudaMalloc(&block, bytes) != cudaSuccess) {
        cudaGetLastError();
        std::lock_guard<std::mutex> lk(s->mu);
        s->used -= bytes;
        return -YORO_ENOMEM;
    }
    Stream st;
    st.live = true;
    st.w = w;
    st.h = h;
    st.fx = fx;
    st.fy = fy;
    st.cx = cx;
    st.cy = cy;
    st.ipd = ipd;
    st.near_ = near_;
    st.far_ = far_;
    st.bytes = bytes;
    st.block = block;
    st.learned = learned != 0;
    for (int i = 0; i < slots; ++i) {
        unsigned char* p = block + per_slot * (size_t)i;
        Slot sl;
        sl.color = p;
        sl.depth = reinterpret_cast<float*>(p + align256(4 * n));
        sl.out = p + 2 * align256(4 * n);
        sl.mask = p + 3 * align256(4 * n);
        sl.zt = learned ? reinterpret_cast<float*>(p + 3 * align256(4 * n) + align256(n)) : nullptr;
        sl.in_flight = false;
        st.slots.push_back(sl);
    }
    std::lock_guard<std::mutex> lk(s->mu);
    s->streams.push_back(std::move(st));
    return (int)s->streams.size() - 1;
}

yoro_status yoro_server_leave(yoro_server s, int stream)
{
    if (!s) return YORO_EINVAL;
    unsigned char* block = nullptr;
    {
        std::unique_lock<std::mutex> lk(s->mu);
        if (stream < 0 || stream >= (int)s->streams.size() || !s->streams[stream].live) return YORO_EINVAL;
        s->cv_done.wait(lk, [&] { return s->streams[stream].pending == 0; });
        Stream& st = s->streams[stream];
        st.live = false;
        block = st.block;
        st.block = nullptr;
        s->used -= st.bytes;
        st.bytes = 0;
        st.slots.clear();
    }
    return cudaFree(block) == cudaSuccess ? YORO_OK : YORO_ECUDA;
}

yoro_status yoro_server_slot(yoro_server s, int stream, int slot, void** color, float** depth, void** out_color,
                             unsigned char** out_hole_mask)
{
    if (!s) return YORO_EINVAL;
    std::lock_guard<std::mutex> lk(s->mu);
    if (stream < 0 || stream >= (int)s->streams.size() || !s->streams[stream].live) return YORO_EINVAL;
    const Stream& st = s->streams[stream];
    if (slot < 0 || slot >= (int)st.slots.size()) return YORO_EINVAL;
    const Slot& sl = st.slots[slot];
    if (color) *color = sl.color;
    if (depth) *depth = sl.depth;
    if (out_color) *out_color = sl.out;
    if (out_hole_mask) *out_hole_mask = sl.mask;
    return YORO_OK;
}

yoro_status yoro_server_submit(yoro_server s, int stream, int slot, unsigned long long tag)
{
    if (!s) return YORO_EINVAL;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        if (stream < 0 || stream >= (int)s->streams.size() || !s->streams[stream].live) return YORO_EINVAL;
        Stream& st = s->streams[stream];
        if (slot < 0 || slot >= (int)st.slots.size() || st.slots[slot].in_flight) return YORO_EINVAL;
        st.slots[slot].in_flight = true;
        ++st.pending;
        ++s->outstanding;
        s->pending.push_back(Request{stream, slot, tag, now_ns(), 0, 0});
    }
    s->cv_work.notify_one();
    return YORO_OK;
}

int yoro_server_poll(yoro_server s, yoro_completion* out, int max)
{
    if (!s || !out || max <= 0) return 0;
    std::lock_guard<std::mutex> lk(s->mu);
    int n = 0;
    while (n < max && !s->done.empty()) {
        out[n++] = s->done.front();
        s->done.pop_front();
    }
    return n;
}

yoro_status yoro_server_drain(yoro_server s, int timeout_ms)
{
    if (!s) return YORO_EINVAL;
    std::unique_lock<std::mutex> lk(s->mu);
    const bool ok = s->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms < 0 ? 0 : timeout_ms),
                                        [&] { return s->outstanding == 0; });
    return ok ? YORO_OK : YORO_ETIMEOUT;
}

yoro_status yoro_server_feed(yoro_server s, int stream, const void* const* colors, const float* const* depths,
                             int nsrc, long long nframes, float hz, unsigned long long tag0)
{
    if (!s || !colors || !depths || nsrc < 1 || nframes < 0 || !(hz >= 0.0f) || !std::isfinite(hz)) return YORO_EINVAL;
    for (int i = 0; i < nsrc; ++i)
        if (!colors[i] || !depths[i]) return YORO_EINVAL;
    std::lock_guard<std::mutex> lk(s->mu);
    if (stream < 0 || stream >= (int)s->streams.size() || !s->streams[stream].live) return YORO_EINVAL;
    if (!s->feeder_started) {
        if (cudaStreamCreateWithFlags(&s->fs, cudaStreamNonBlocking) != cudaSuccess) {
            cudaGetLastError();
            return YORO_ECUDA;
        }
        try {
            s->feeder = std::thread([s] { s->feed_loop(); });
        } catch (...) {
            cudaStreamDestroy(s->fs);
            s->fs = nullptr;
            return YORO_ENOMEM;
        }
        s->feeder_started = true;
    }
    FeedJob jb;
    jb.stream = stream;
    jb.colors.assign(colors, colors + nsrc);
    jb.depths.assign(depths, depths + nsrc);
    jb.remaining = nframes;
    jb.next = 0;
    jb.period_ns = hz > 0.0f ? 1e9 / (double)hz : 0.0;
    jb.due_ns = now_ns();
    jb.tag = tag0;
    s->jobs.push_back(std::move(jb));
    s->cv_done.notify_all();
    return YORO_OK;
}

yoro_status yoro_server_feed_stop(yoro_server s)
{
    if (!s) return YORO_EINVAL;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        for (FeedJob& jb : s->jobs) jb.remaining = 0;
        s->jobs.clear();
    }
    s->cv_done.notify_all();
    return YORO_OK;
}

yoro_status yoro_server_set_inpainter(yoro_server s, yoro_unet u)
{
    if (!s) return YORO_EINVAL;
    std::lock_guard<std::mutex> lk(s->mu);
    s->inpainter = u;
    return YORO_OK;
}

yoro_status yoro_server_pause(yoro_server s, int paused)
{
    if (!s || (paused != 0 && paused != 1)) return YORO_EINVAL;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->paused = paused != 0;
    }
    s->cv_work.notify_all();
    return YORO_OK;
}

int yoro_server_cancel(yoro_server s, int stream)
{
    if (!s) return -YORO_EINVAL;
    int n = 0;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        if (stream < 0 || stream >= (int)s->streams.size() || !s->streams[stream].live) return -YORO_EINVAL;
        Stream& st = s->streams[stream];
        const long long t = now_ns();
        for (auto it = s->pending.begin(); it != s->pending.end();) {
            if (it->stream != stream) {
                ++it;
                continue;
            }
            yoro_completion c;
            c.stream = it->stream;
            c.slot = it->slot;
            c.tag = it->tag;
            c.submit_ns = it->submit_ns;
            c.launch_ns = 0;
            c.done_ns = t;
            c.batch_frames = 0;
            c.status = YORO_ECANCELED;
            c.inpainted = 0;
            s->done.push_back(c);
            st.slots[it->slot].in_flight = false;
            --st.pending;
            --s->outstanding;
            ++n;
            it = s->pending.erase(it);
        }
    }
    s->cv_done.notify_all();
    return n;
}

size_t yoro_server_memory_used(yoro_server s)
{
    if (!s) return 0;
    std::lock_guard<std::mutex> lk(s->mu);
    return s->used;
}

}  // extern "C"
