/*
 * yoro_server.h — serving loop of the second-eye synthesis library (libyoro.so).
 *
 * A library service with no counterpart in the paper: many headset streams share one
 * GPU.  Each admitted stream keeps resident frame slots in device memory (left-eye
 * color and depth, right-eye color and hole mask), admitted against a device-memory
 * budget.  A client (the renderer of a stream) writes a left eye into one of its slots
 * and submits it; a scheduler thread owned by the server runs continuous batching: the
 * moment the previous launch completes, every frame submitted meanwhile (up to a batch
 * limit) goes into the next yoro_synthesize_batch launch, so a frame waits at most for
 * one batch in flight.  Each frame's result is the same as yoro_synthesize's for that
 * frame, whatever else shares its batch.
 *
 * Threading: every function may be called from any host thread.  A slot must not be
 * written or resubmitted between its submit and its completion (poll).
 */
#ifndef YORO_SERVER_H
#define YORO_SERVER_H

#include <stddef.h>

#include "yoro.h"
#include "yoro_unet.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct yoro_server_ctx* yoro_server;

/* One completed frame. Times are host steady-clock nanoseconds. */
typedef struct {
    int stream;                  /* stream id from yoro_server_admit                        */
    int slot;                    /* slot that held the frame                                */
    unsigned long long tag;      /* the caller's tag from yoro_server_submit                */
    long long submit_ns;         /* when yoro_server_submit queued it                       */
    long long launch_ns;         /* when the batch that held it was launched                */
    long long done_ns;           /* when the scheduler saw that batch complete              */
    int batch_frames;            /* frames in that batch (0: cancelled before a launch)     */
    yoro_status status;          /* YORO_OK, the batch launch's error, or YORO_ECANCELED    */
    int inpainted;               /* 1: the learned inpainter repainted the holes; 0: the
                                    paper's fill (plain streams, no inpainter, or fallback) */
} yoro_completion;

/*
 * Create a server on the current device with a budget of device memory for the streams'
 * resident slots and at most max_batch frames per launch (1..4096).  Starts the
 * scheduler thread.  Returns NULL on error (yoro_last_create_error() tells why:
 * YORO_EINVAL for a zero budget or a bad max_batch, YORO_ECUDA, YORO_ENOMEM).
 */
yoro_server yoro_server_create(size_t memory_budget_bytes, int max_batch);

/* Stop the scheduler after the frames already submitted, free every stream's slots and
 * the server.  NULL is accepted. */
void yoro_server_destroy(yoro_server s);

/*
 * Admit a stream of w x h frames of a stereo camera (parameters as yoro_create; frames
 * must not be wider than yoro_max_fused_width()) with `slots` resident frame slots
 * (1..64).  Returns the stream id (>= 0), or the negated status: -YORO_EINVAL for bad
 * arguments, -YORO_ETOOBIG for a too wide frame, -YORO_ENOMEM if the slots would exceed
 * the budget or the device allocation fails (the caller may retry after a stream has
 * left).
 */
int yoro_server_admit(yoro_server s, int w, int h, float fx, float fy, float cx, float cy, float ipd,
                      float near_, float far_, int slots);

/*
 * yoro_server_admit() with a choice of hole fill: learned = 1 gives each slot a warped-
 * depth buffer too (4 more bytes per pixel against the budget), and the frames of the
 * stream are repainted by the server's inpainter (yoro_server_set_inpainter) after the
 * synthesis; learned = 0 is yoro_server_admit().  A learned frame keeps the paper's fill
 * (its fallback) when no inpainter is set or the inpainter does not take its size; its
 * completion says which (inpainted).
 */
int yoro_server_admit_ex(yoro_server s, int w, int h, float fx, float fy, float cx, float cy, float ipd,
                         float near_, float far_, int slots, int learned);

/*
 * The learned inpainter (yoro_unet.h) that repaints the frames of learned streams, or
 * NULL for none.  The server does not own it: keep it alive, and do not use it on other
 * streams, until the server is destroyed or another one (or NULL) is set and the frames
 * submitted before have completed (drain).  Takes effect from the next batch.
 */
yoro_status yoro_server_set_inpainter(yoro_server s, yoro_unet u);

/*
 * paused = 1: launch nothing new (frames already launched complete; frames submitted
 * wait); paused = 0: resume.  A headset that is taken off, or a test of what waits.
 */
yoro_status yoro_server_pause(yoro_server s, int paused);

/*
 * Cancel the frames of `stream` that are queued and not launched: each completes at once
 * with YORO_ECANCELED (batch_frames 0) and its slot is free again; frames already in a
 * batch complete normally.  Returns how many were cancelled, or the negated status
 * (-YORO_EINVAL for an unknown stream).
 */
int yoro_server_cancel(yoro_server s, int stream);

/*
 * Feed a stream from device memory without a host loop: the server's feeder thread
 * copies source frame i % nsrc (colors[i]: w*h*4 bytes, depths[i]: w*h floats, device
 * pointers the caller keeps valid until the job ends) into a free slot of the stream and
 * submits it, nframes times, with tags tag0, tag0 + 1, ...; hz > 0 paces the frames at
 * that rate, hz = 0 sends each as soon as a slot is free.  Returns at once; completions
 * arrive through yoro_server_poll as for yoro_server_submit.  Jobs of several streams run
 * side by side.  A stream fed this way must not also be submitted to by the caller.
 */
yoro_status yoro_server_feed(yoro_server s, int stream, const void* const* colors, const float* const* depths,
                             int nsrc, long long nframes, float hz, unsigned long long tag0);

/* End every feeding job (frames already submitted complete normally). */
yoro_status yoro_server_feed_stop(yoro_server s);

/* Remove a stream: waits until its submitted frames are done, then frees its slots.
 * Its completions stay available to yoro_server_poll. */
yoro_status yoro_server_leave(yoro_server s, int stream);

/* Device pointers of a slot (layout as yoro_synthesize: RGBA8 color, f32 depth, RGBA8
 * out_color, u8 out_hole_mask, tightly packed rows, 256-byte aligned). */
yoro_status yoro_server_slot(yoro_server s, int stream, int slot, void** color, float** depth, void** out_color,
                             unsigned char** out_hole_mask);

/* Queue the frame in `slot` of `stream` (its inputs written and synchronised by the
 * caller).  Returns at once.  YORO_EINVAL for an unknown stream or slot, or a slot still
 * in flight. */
yoro_status yoro_server_submit(yoro_server s, int stream, int slot, unsigned long long tag);

/* Move up to max completed frames (oldest first) into out; returns how many. */
int yoro_server_poll(yoro_server s, yoro_completion* out, int max);

/* Block until every submitted frame is done (or the timeout in milliseconds passes);
 * YORO_OK, or YORO_ETIMEOUT if the timeout passed first. */
yoro_status yoro_server_drain(yoro_server s, int timeout_ms);

/* Bytes of the budget in use by admitted streams. */
size_t yoro_server_memory_used(yoro_server s);

#ifdef __cplusplus
}
#endif

#endif /* YORO_SERVER_H */
