/*
 * canny.h -- C ABI of libcanny, a GB300 (sm_103a) Canny edge detector.
 *
 * The operation is the four-step pipeline of H. Mogale, "High Performance
 * Canny Edge Detector using Parallel Patterns for Scalability on Modern
 * Multicore Processors", Sec. 2.2.1 (Algorithm 1; Steps 1-4):
 *   Step 1  Gaussian noise filter;
 *   Step 2  Sobel gradient: strength and direction;
 *   Step 3  non-maximum suppression;
 *   Step 4  hysteresis: strength above the upper threshold is an edge, below
 *           the lower one is not, in between is an edge only if connected to
 *           an edge pixel above the upper threshold.
 * The paper states the problem as: a grayscale image, a smoothing parameter
 * and two thresholds in; an edge map out.
 *
 * Constants the paper leaves open are fixed as follows.
 *   Integer path (CANNY_PATH_INT, bit-exact):
 *     - 5x5 binomial Gaussian (1,4,6,4,1)^2 / 256, rounded half up;
 *     - replicate (clamp-to-edge) border for the image and the smoothed image;
 *     - Sobel Gx (x right), Gy (y down), strength Gx^2 + Gy^2;
 *     - direction: 4 sectors with tan(22.5 deg) as 13573 / 2^15;
 *     - suppression keeps a pixel that beats its negative-side neighbour
 *       strictly and its positive-side neighbour or ties it; neighbours
 *       outside the image count as 0;
 *     - thresholds compared squared and strictly: weak if low^2 < G^2 <= high^2,
 *       strong if G^2 > high^2; low and high must be integers in [0, 2^15);
 *     - hysteresis through 8-connected weak/strong pixels.
 *   Float path (CANNY_PATH_F32): sigma-parametrised separable Gaussian of odd
 *     size ksize (taps exp(-k^2 / 2 sigma^2), normalised), float32 Sobel and
 *     L2 strength, tan(22.5 deg) as 0.41421356f, thresholds low/high given as
 *     fractions of the image's largest strength.
 *
 * Memory and ownership. All image pointers are device pointers (cudaMalloc,
 * torch tensors) unless a function says "host". The caller owns every image
 * buffer and the stream; the context owns its scratch (hysteresis tile state
 * and worklists, the float path's strength buffer, the CUDA graph). The input
 * is never written. The output must not overlap the input. Images are
 * row-major uint8, row stride = pitch bytes (pitch >= width). Only the first
 * `w` bytes of each output row are written; output values are 0 or 255.
 *
 * Errors. Functions return a canny_status and never abort. Argument errors
 * are reported synchronously, before any work is queued. Launch failures
 * return CANNY_ECUDA. Work is queued asynchronously on the given stream
 * (a cudaStream_t passed as void*; NULL is the legacy default stream);
 * an error raised while that work runs (including CANNY_ENOCONVERGE, the
 * hysteresis pass cap) is reported by canny_get_stats(), which synchronises.
 *
 * Threads. A context serves one stream at a time: calls that share a context
 * must be ordered on the same stream. Separate contexts are independent.
 */
#ifndef CANNY_H
#define CANNY_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    CANNY_OK = 0,
    CANNY_EINVAL = 1,          /* bad argument: null pointer, size, pitch, threshold */
    CANNY_ENOMEM = 2,          /* device or pinned allocation failed */
    CANNY_ECUDA = 3,           /* a CUDA call or kernel launch failed */
    CANNY_ENOCONVERGE = 4,     /* hysteresis hit its pass cap before its fixpoint */
    CANNY_EUNSUPPORTED = 5     /* request outside what this build supports */
} canny_status;

enum { CANNY_PATH_INT = 0, CANNY_PATH_F32 = 1 };

typedef struct {
    int path;          /* CANNY_PATH_INT or CANNY_PATH_F32 */
    float sigma;       /* float path: Gaussian sigma (> 0); ignored by the integer path */
    int ksize;         /* float path: odd kernel size in [3, 31]; the integer path uses 5 */
    float low, high;   /* integer path: absolute strengths (integers, compared squared);
                          float path: fractions of the largest strength; low <= high */
    int max_passes;    /* cap on global hysteresis passes; 0 = automatic */
} canny_params;

/* One image of a pitched run or of a batch. */
typedef struct {
    const uint8_t *d_in;   /* device, h rows of in_pitch bytes */
    uint8_t *d_out;        /* device, h rows of out_pitch bytes; not overlapping d_in */
    int w, h;              /* pixels; w == 0 or h == 0 is an empty image (nothing written) */
    int in_pitch, out_pitch;
} canny_image;

/* Counters of the most recent run on a context (read after synchronising). */
typedef struct {
    int64_t images;            /* images in the last run */
    int64_t pixels;            /* pixels in the last run */
    int64_t tiles;             /* 32x32 hysteresis tiles in the last run */
    int64_t hyst_passes;       /* global hysteresis passes the last run took */
    int64_t hyst_tiles_visited;/* tile visits summed over those passes */
    int64_t pending_tiles;     /* tiles left with unresolved weak pixels after the local fill */
    int32_t status;            /* canny_status of the last run's device work */
    int32_t reserved;
} canny_stats;

typedef struct canny_ctx canny_ctx;

/* Fill *p with the defaults: integer path, low 40, high 100, sigma 1.4, ksize 7. */
canny_status canny_params_default(canny_params *p);

/*
 * Set-up for Steps 1-4 (Sec. 2.2.1): create a context for images of at most max_w x max_h pixels (the pixel
 * budget max_w * max_h also bounds the total pixels of one canny_run_batch
 * call). Allocates the scratch on the current device. Returns CANNY_EINVAL for
 * non-positive sizes or invalid params, CANNY_ENOMEM if allocation fails.
 */
canny_status canny_create(int max_w, int max_h, const canny_params *p, canny_ctx **out);

/* Free the context and its scratch. Synchronises the device first. NULL is a no-op. */
void canny_destroy(canny_ctx *ctx);

/*
 * Steps 1-4 (Sec. 2.2.1, Algorithm 1): edge map of one max_w x max_h image with
 * tight rows (pitch = max_w); d_in and d_out are device buffers of
 * max_w * max_h bytes. On the integer path the classes of Steps 1-3 and the
 * double threshold pass from the stencil to the hysteresis as two bits per
 * pixel in the context's tile scratch (0.25 byte per pixel); d_out is written
 * once, with the final edge map. Asynchronous on stream.
 */
canny_status canny_run(canny_ctx *ctx, const uint8_t *d_in, uint8_t *d_out, void *stream);

/*
 * Steps 1-4 (Sec. 2.2.1): edge map of one image of any size up to the
 * context's, with its own pitches.
 * An input whose base address or pitch is not a multiple of 16 bytes is first
 * copied on the device into a 16-byte pitched staging buffer of the context
 * (allocated on first need, which synchronises the device once, and kept until
 * canny_destroy); if that allocation fails the image is read directly instead.
 * Same for canny_run (pitch max_w) and canny_run_host.
 */
canny_status canny_run_pitched(canny_ctx *ctx, const canny_image *img, void *stream);

/*
 * Steps 1-4 over many images at once (Sec. 2.2.2: the work of all images
 * shared out to the cores as one pool of tasks): edge maps of n images of any
 * sizes (total pixels at most max_w * max_h, the context's pixel budget) in
 * one launch sequence: every stage runs once over the tiles of all images. The image descriptors are read from host
 * memory before the call returns. Outputs equal n separate canny_run_pitched
 * calls byte for byte.
 */
canny_status canny_run_batch(canny_ctx *ctx, int n, const canny_image *imgs, void *stream);

/*
 * Steps 1-4 (Sec. 2.2.1) end to end on host buffers: copies h_in (host, h rows of in_pitch bytes)
 * to the device, runs the pipeline and copies the edge map back to h_out (host,
 * h rows of out_pitch bytes); returns after the stream has been synchronised.
 * Pinned (page-locked) host buffers give the fastest copies. Device buffers for
 * the copies are owned by the context.
 */
canny_status canny_run_host(canny_ctx *ctx, const uint8_t *h_in, int in_pitch, uint8_t *h_out,
                            int out_pitch, int w, int h, void *stream);

/*
 * A sequence of n frames of one size w x h on host buffers (video): frame i is
 * read from h_in[i] (h rows of in_pitch bytes) and its edge map written to
 * h_out[i] (h rows of out_pitch bytes). The paper points to real-time video
 * processing on multicore processors (Sec. 2.1, ref. [14]) and to high
 * resolution image and video work (Sec. 4); here consecutive frames overlap:
 * the upload of frame i+1, the pipeline on frame i and the download of frame
 * i-1 run at the same time on three streams, and each frame's pipeline is one
 * replay of a CUDA graph built once per frame size (two device slots).
 * Each output equals canny_run_host on that frame. Pinned host buffers are
 * needed for the copies to overlap. Returns after the last edge map is in
 * h_out; CANNY_ENOCONVERGE if any frame reached the hysteresis pass cap.
 * Device buffers, streams and graphs are owned by the context. The work on
 * `stream` (the pipelines) starts after what is already queued on it.
 */
canny_status canny_run_frames(canny_ctx *ctx, int n, const uint8_t *const *h_in, int in_pitch,
                              uint8_t *const *h_out, int out_pitch, int w, int h, void *stream);

/*
 * Steps 1-3 and the double threshold of Step 4 (Sec. 2.2.1) only: the class
 * map before the connectivity search,
 * 0 (none), 1 (weak) or 2 (strong) per pixel, into img->d_out.
 */
canny_status canny_classify(canny_ctx *ctx, const canny_image *img, void *stream);

/*
 * Step 4's connectivity search only (Sec. 2.2.1; weak pixels kept when
 * 8-connected to a strong one): img->d_in holds a class map (0 none, 1 weak, 2 strong; other
 * values count as strong); the 0/255 edge map goes to img->d_out.
 */
canny_status canny_hysteresis(canny_ctx *ctx, const canny_image *img, void *stream);

/*
 * Float path, Steps 1-2 only (Sec. 2.2.1 Step 2, "gradient strength"): the
 * strength M (float32, row stride d_mag_pitch floats) of img into d_mag, and the
 * image's largest strength into *d_max (device float), as computed by the
 * float pipeline's own first pass (M = sqrt_rn(Gx^2 + Gy^2) per pixel). The
 * context must use CANNY_PATH_F32.
 */
canny_status canny_magnitude_f32(canny_ctx *ctx, const canny_image *img, float *d_mag,
                                 int d_mag_pitch, float *d_max, void *stream);

/* Device time per stage, summed over the runs since the last canny_read_timing. */
typedef struct {
    int64_t runs;          /* runs timed */
    double reset_ms;       /* clearing the hysteresis worklist state */
    double stencil_ms;     /* Steps 1-3 + thresholds and the per-tile fill (integer path: the fused
                              stencil and the tile-fill kernel; float path: both passes, the second
                              fused with the fill) */
    double local_ms;       /* hysteresis: per-tile fill of canny_hysteresis (a class map input) */
    double global_ms;      /* hysteresis: global passes */
    double total_ms;       /* first stage start to last stage end, summed over runs */
} canny_timing;

/*
 * Turn per-stage timing on (enable != 0) or off. While on, every canny_run /
 * canny_run_pitched records CUDA events on its stream around each stage
 * (at most 4096 runs between reads; later runs are not timed).
 */
canny_status canny_enable_timing(canny_ctx *ctx, int enable);

/* Synchronise, sum the stage times of the runs timed since the last read into *out, reset. */
canny_status canny_read_timing(canny_ctx *ctx, canny_timing *out);

/*
 * Launch configuration of the fused integer kernel: rows per unit of work
 * (band: 32, 64, 160 or 256; taller bands cut halo work, shorter ones balance
 * small images better; 0, the default: 32 or 64 rows chosen per image size for
 * single images, 64 for batches) and, for batches, ctas_per_sm: 0 (the default) launches one
 * CTA per (image, strip, band) unit and lets the hardware schedule them, 1..32
 * launches that many persistent CTAs per SM that pop units from a device
 * counter. direct_loads = 1 reads
 * inputs whose base or pitch is not a multiple of 16 bytes directly instead of
 * repitching them into staging first (slower; no staging memory); 0 or 1.
 *
 * Schedule of the global hysteresis passes (Step 4's connectivity search):
 * chase_budget is how many further tiles a weak chain may be followed into
 * within a pass before the rest is left to the next one (1..4096; 0, the
 * default, takes 16 in a cooperative launch, 64 in a loop of one launch per
 * pass, and 4 for single images on the float path, whose long weak chains the
 * union-find stage below resolves sooner than longer chases). Where the passes run in one cooperative launch (single images;
 * batches with batch_passes = 1), work left after the first pass is resolved at
 * once by union-find over tile-border components when that pass's worklist held
 * at most 32768 tiles, and by further passes otherwise. batch_passes picks how
 * a batch graph runs the passes: 0 (the default) a graph while-loop of one
 * launch per pass, 1 one cooperative kernel node; 1 falls back to 0 where the
 * device cannot hold that grid. Every setting gives the same edge map.
 */
typedef struct {
    int band;
    int ctas_per_sm;
    double ms;        /* canny_autotune_batch: measured time of one batch run */
    int from_cache;   /* canny_autotune_batch: 1 if read from the cache file */
    int direct_loads;
    int chase_budget;
    int batch_passes;
} canny_tuning;

/* Apply a configuration; CANNY_EINVAL for an unsupported band or CTA count. */
canny_status canny_set_tuning(canny_ctx *ctx, const canny_tuning *t);
canny_status canny_get_tuning(const canny_ctx *ctx, canny_tuning *out);

/*
 * How the work is split (Sec. 2.2.2: the split of tasks over cores decides the
 * load balance): pick the configuration for batches like `imgs` (integer path): look up the
 * size class (device, image count and mean area in octaves) in cache_path
 * (JSON lines; NULL for none); if absent, time candidates on this batch in
 * three stages, each keeping the best of the one before: tile shape (band x
 * ctas_per_sm), then the halo layout of unaligned inputs (direct_loads 0/1,
 * only when the batch has such an input), then the pass schedule
 * (chase_budget x batch_passes). Each candidate runs the batch three times
 * (outputs are overwritten with the same edge maps). The winner is appended to
 * cache_path and applied. Synchronous.
 */
canny_status canny_autotune_batch(canny_ctx *ctx, int n, const canny_image *imgs, void *stream,
                                  const char *cache_path, canny_tuning *out);

/* Copy the counters of the last run into *out. Synchronises the context's last stream. */
canny_status canny_get_stats(canny_ctx *ctx, canny_stats *out);

/*
 * Steps 1-4 (Sec. 2.2.1), integer pipeline without any device allocation. The
 * paper has no counterpart for the allocation rule:
 * this entry point exists for callers that cannot call cudaMalloc -- code that
 * runs under a device-memory budget held entirely by another allocator (a
 * framework's caching allocator, a fixed arena), or a frame loop in which the
 * implicit device synchronisation of cudaMalloc/cudaFree is not allowed.
 *
 * Same result as canny_run_pitched on an integer-path context with thresholds
 * low/high (integers, 0 <= low <= high < 2^15). The caller passes the device
 * input and output as for canny_run_pitched; no context is needed. The
 * hysteresis scratch is one fixed device array in the library (about 7 MB,
 * held on every GPU that loads the library until the process exits), so the
 * image may have at most 16384 tiles of 32x32 pixels (16.8 Mpixel, e.g.
 * 4096 x 4096); larger images return CANNY_EUNSUPPORTED before any work is
 * queued. Every call shares that array: calls that overlap on the GPU (other
 * streams, other threads) race and must be serialised by the caller. The first
 * call on each device looks up the array's device address (set-up, once per
 * device). The global hysteresis passes run in one cooperative launch where
 * the device allows, otherwise (or if the device refuses that grid) the host
 * drives them, one pass at a time. Either way the call reads the result's
 * status back, so it synchronises the stream before it returns.
 */
canny_status canny_run_noalloc(const uint8_t *d_in, int in_pitch, uint8_t *d_out, int out_pitch,
                               int w, int h, int low, int high, void *stream);

/* One request of a served trace. */
typedef struct {
    int w, h;               /* image size */
    const uint8_t *h_in;    /* host, h rows of h_pitch bytes; page-locked, 16-byte aligned buffers with
                               h_pitch == w are read by one kernel per batch, others by copy-engine copies */
    int h_pitch;
    uint8_t *h_out;         /* host buffer for the 0/255 edge map (same rule as h_in), or NULL to leave
                               it on the device */
    int out_pitch;
    double arrival_s;       /* arrival time, seconds after the start of the run; non-decreasing */
} canny_request;

typedef struct {
    double memory_budget_bytes;   /* device memory for the requests' inputs and outputs */
    int streams;                  /* batches in flight at once (>= 1) */
    int max_batch_images;         /* images per batch, at most (1 .. 65535) */
    int64_t max_batch_pixels;     /* pixels per batch, at most (>= the largest request) */
    int serial;                   /* 1: one request at a time through canny_run_pitched (baseline) */
    int low, high;                /* integer-path thresholds */
    int band, ctas_per_sm;        /* fused-kernel configuration (band 0: defaults) */
} canny_serve_config;

typedef struct {
    int64_t completed;
    double wall_s;                /* first arrival to last completion */
    double delivered_mpx_s;       /* pixels served / wall_s */
    double p50_ms, p99_ms, max_ms;/* latency: completion (event observed) minus arrival */
    int64_t batches;
    double mean_batch_images;
    int64_t peak_bytes;           /* most arena bytes in use at once */
    int64_t deferrals;            /* admissions put off because the arena had no room */
} canny_serve_report;

/*
 * Steps 1-4 (Sec. 2.2.1) as a service: serve a request trace in real time with
 * continuous batching (integer path).
 * Requests arriving while earlier ones run are admitted in arrival order as
 * soon as the memory budget has room for their input and output buffers;
 * the idle streams share the admitted, not-yet-running requests in arrival
 * order, each taking about an equal part of their pixels as one
 * canny_run_batch (a lone idle stream takes them all, up to the batch
 * limits), so batches of later arrivals overlap earlier ones on the GPU.
 * Each result equals the request's canny_run_pitched result. Writes the
 * per-request latencies (ms) to latency_ms if not NULL. Synchronous: returns
 * when every request has completed. The budget is allocated once per call.
 * CANNY_EINVAL if a request's input and output buffers (16-byte pitched rows)
 * alone exceed the budget; CANNY_ENOMEM if the budget or the streams' buffers
 * cannot be allocated.
 */
canny_status canny_serve(const canny_serve_config *cfg, int n, const canny_request *reqs, double *latency_ms,
                         canny_serve_report *out);

/*
 * Test hooks for failure detection, with no GPU fault involved. Counts of
 * events that go wrong from now on (process-wide; each call replaces the
 * pending counts; CANNY_EINVAL if one is negative):
 *   device_allocations  the next device or pinned-host allocations made by the
 *                       library (contexts, scratch, staging, maps, serving
 *                       budget) fail as if out of memory;
 *   arena_admissions    the next request admissions of canny_serve find no
 *                       room in its budget (the request waits for the next
 *                       attempt);
 *   stalled_barriers    the next single-image runs start their global
 *                       hysteresis passes with a grid barrier that can never
 *                       complete: its bounded wait runs out (after a second
 *                       of GPU time) and the run reports CANNY_ECUDA through
 *                       canny_get_stats; the context stays usable;
 *   host_driven_passes  the next single-image runs (canny_run,
 *                       canny_run_pitched, canny_run_noalloc) drive their
 *                       global hysteresis passes from the host, one launch
 *                       and one read of the control block per pass, as when
 *                       the device refuses the cooperative grid.
 */
typedef struct {
    int device_allocations;
    int arena_admissions;
    int stalled_barriers;
    int host_driven_passes;
} canny_fault_injection;

canny_status canny_inject_faults(const canny_fault_injection *f);

/* Static, human-readable message for a status. */
const char *canny_strerror(canny_status s);

#ifdef __cplusplus
}
#endif
#endif /* CANNY_H */
