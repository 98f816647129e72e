/*
 * fasthog_server.h -- a request server over the detection path of fasthog.h:
 * continuous batching of images of any size on one GPU.
 *
 * The paper has no counterpart: it runs the detector on one image at a time.
 * This layer sits above the per-image calls (hog_cell_hist_fused or
 * hog_bin_map + hog_integral + hog_cell_hist, then hog_window_score and
 * hog_detect) and runs many images at once.  Requests are admitted while
 * others are still on the GPU, as long as a slot (one CUDA stream) is free
 * and the request's buffers fit in the device-memory budget; their work
 * overlaps on the device.  Every admitted request has buffers of its own, so
 * its result does not depend on what else is running.
 *
 * Memory.  hog_server_create allocates everything the server will use: one
 * device arena of `budget_bytes` (requests' image, cell map and scores, plus
 * bin map, integral images and their workspace when the path is not fused),
 * the gradient table and the weights (resident for the server's life), and
 * per slot a stream, an event, a detection workspace sized for the largest
 * request (zero-filled once; every request leaves it ready for the next) and
 * a page-locked host buffer that the GPU writes the detection list and its
 * count into directly.  Submit and
 * poll allocate nothing: a request's buffers are carved out of the arena
 * (first fit, 256-byte aligned) and returned to it when the request
 * completes.
 *
 * Threads.  Without the dispatcher thread (below) a server is used by one
 * host thread at a time; calls on one server from several threads must be
 * serialised by the caller.  With it, enqueue, collect and release may come
 * from any thread.  All calls run on the device that was current at
 * hog_server_create (they switch to it and back if another device is
 * current).
 *
 * Errors follow fasthog.h: HOG_ERR_ARG for bad arguments (nothing is
 * enqueued), HOG_ERR_CUDA with hog_last_cuda_error() for a failed CUDA call.
 */
#ifndef FASTHOG_SERVER_H
#define FASTHOG_SERVER_H

#include "fasthog.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct hog_server hog_server; /* opaque */

typedef struct {
    int n_bins;          /* N_b, 1..64 */
    int cell;            /* cell side in pixels */
    int stride;          /* scan step in pixels; cell % stride == 0 */
    int cells_x;         /* window width in cells */
    int cells_y;         /* window height in cells */
    int w_dtype;         /* HOG_F32, HOG_BF16 or HOG_I8 (scores are int32 for HOG_I8, else float) */
    float bias;          /* added to every window score */
    float thr;           /* a window is detected when its score >= thr */
    int fused;           /* 1: hog_cell_hist_fused; 0: the three separate calls, which keep each
                            request's bin map and integral images on the device; -1: fused where
                            hog_cell_hist_fused supports the parameters */
    int ii_dtype;        /* integral-image type of the separate calls: HOG_I32 or HOG_U16 */
    int n_slots;         /* requests on the GPU at once (one stream each), 1..64 */
    size_t budget_bytes; /* device memory for the requests' buffers */
    int max_W, max_H;    /* largest image accepted; sizes each slot's host detection buffer */
    int image_in_place;  /* 1: a request whose image is page-locked host memory mapped into the
                            device's address space (cudaHostAlloc, cudaHostRegister, or PyTorch's
                            pinned memory) is read in place by its first kernel, so its bytes
                            cross to the GPU inside that kernel and no copy is enqueued; other
                            images are copied in.  0: every image is copied in first. */
} hog_server_config;

typedef struct {
    int32_t rid;          /* the id given to hog_server_submit (also each detection's `image`) */
    int32_t status;       /* HOG_OK, or HOG_ERR_CUDA if the request's work failed on the GPU */
    int32_t count;        /* number of windows with score >= thr; all of them are in dets */
    int32_t token;        /* hand back with hog_server_release when done with dets */
    int32_t W, H;         /* the request's image size */
    const hog_det* dets;  /* `count` detections in row-major window order, in HOST memory owned
                             by the server, valid until hog_server_release(token) */
} hog_server_result;

/* Create a server.  `w` is a HOST array of cells_y * cells_x * n_bins
 * weights of type cfg->w_dtype, in the feature order of hog_window_score;
 * it is copied.  Builds the gradient table, allocates all memory, and
 * synchronises the device once before returning.  *out is NULL on error. */
hog_status hog_server_create(const hog_server_config* cfg, const void* w, hog_server** out);

/* Wait for every request still on the GPU, then free everything.  NULL is
 * accepted (HOG_OK). */
hog_status hog_server_destroy(hog_server* s);

/* Arena bytes a request of this size holds while on the GPU (0 for an
 * invalid size). */
size_t hog_server_request_bytes(const hog_server* s, int W, int H, int channels);

/* Submit one request: `img` is a HOST image of H rows of W * channels bytes
 * (channels 1 = gray, 3 = interleaved RGB), rows contiguous.  Page-locked
 * memory lets the copy overlap other work; pageable memory also works, with
 * the copy staged by the driver.  The image must stay unchanged until the
 * request's result has been returned by hog_server_poll.
 *
 * *admitted = 1: the request is on the GPU.  *admitted = 0 (HOG_OK): no slot
 * is free or its buffers do not fit in the arena right now; submit it again
 * after a poll has returned results.  HOG_ERR_ARG: a bad argument, a size
 * above max_W x max_H, or a request that needs more than the whole budget;
 * it can never be admitted. */
hog_status hog_server_submit(hog_server* s, int32_t rid, const uint8_t* img, int W, int H, int channels,
                             int* admitted);

/* Collect completed requests without blocking: writes up to max_out results
 * to `out` (host memory) and their number to *n_out.  A returned request's
 * arena memory is free again at once; its slot is free again after
 * hog_server_release. */
hog_status hog_server_poll(hog_server* s, hog_server_result* out, int max_out, int* n_out);

/* Give back the detection buffer of a result returned by hog_server_poll. */
hog_status hog_server_release(hog_server* s, int32_t token);

/* Requests on the GPU, arena bytes they hold, and slots that are neither on
 * the GPU nor awaiting release.  Any pointer may be NULL.  HOG_ERR_UNSUPPORTED
 * while the dispatcher thread runs (it owns these counts then). */
hog_status hog_server_stats(const hog_server* s, int* in_flight, size_t* bytes_in_use, int* free_slots);

/*
 * The server's own dispatcher thread (optional).  hog_server_start launches a
 * host thread that admits queued requests in arrival order (first in, first
 * out) as soon as a slot is free and their buffers fit, and watches the
 * requests on the GPU; so admission and completion never wait for a call
 * from the caller, and a stall of the caller's thread delays neither.
 * While it runs, use hog_server_enqueue, hog_server_collect and
 * hog_server_release (from any thread) instead of hog_server_submit and
 * hog_server_poll.  hog_server_stop waits until every queued request has
 * completed, then joins the thread; the results it left stay collectable.
 * hog_server_destroy stops a running dispatcher first.
 *
 * Timestamps are nanoseconds of the steady clock that hog_server_clock_ns
 * reads (CLOCK_MONOTONIC).
 */
typedef struct {
    hog_server_result r;   /* as hog_server_poll returns it; release r.token when done with r.dets */
    int64_t t_enqueue_ns;  /* when hog_server_enqueue queued the request (its arrival) */
    int64_t t_admit_ns;    /* when the dispatcher put its work on the GPU */
    int64_t t_done_ns;     /* when the dispatcher saw its work complete (detections in host memory) */
} hog_server_timed_result;

hog_status hog_server_start(hog_server* s);
hog_status hog_server_stop(hog_server* s);
/* Queue one request (arguments as hog_server_submit; the image must stay
 * unchanged until its result is collected).  Never waits for the GPU.
 * HOG_ERR_ARG for a request that can never be admitted (nothing is queued);
 * HOG_ERR_UNSUPPORTED when the dispatcher is not running. */
hog_status hog_server_enqueue(hog_server* s, int32_t rid, const uint8_t* img, int W, int H, int channels);
/* Completed requests, oldest first: up to max_out of them to `out` (host
 * memory), their number to *n_out.  Never blocks on the GPU. */
hog_status hog_server_collect(hog_server* s, hog_server_timed_result* out, int max_out, int* n_out);
int64_t hog_server_clock_ns(void);
/* Pauses of the dispatcher thread since hog_server_start: stretches of more
 * than 1 ms between two turns of its loop.  A turn only queries events and
 * enqueues asynchronous work, so such a stretch means the thread was not
 * running (the operating system or the host paused the process); requests in
 * flight or queued then wait whatever the GPU does.  Writes the [start, end]
 * stamps (hog_server_clock_ns) of the most recent min(max_n, kept) pauses,
 * oldest first (the last 4096 are kept), and the number of pauses since
 * hog_server_start to *n.  Callable from any thread while the dispatcher
 * runs, and after it stopped.  HOG_ERR_ARG for a NULL server or n, a negative
 * max_n, or NULL stamp arrays with max_n > 0. */
hog_status hog_server_pauses(hog_server* s, int64_t* start_ns, int64_t* end_ns, int max_n, int* n);

#ifdef __cplusplus
}
#endif

#endif /* FASTHOG_SERVER_H */
