/*
 * kq.h -- C ABI of the GB300 exact k-means colour quantizer (Weighted Sort-Means,
 * M. E. Celebi, "Improving the Performance of K-Means for Color Quantization",
 * Image and Vision Computing 29(4), 2011; arXiv:1101.0395).
 *
 * The four steps of the method, each one call:
 *   kq_histogram  unique colours with integer weights          (Section 2.2, items 1-2)
 *   kq_seed       initial centres by a generic scheme           (Section 2.3)
 *   kq_lloyd      weighted Lloyd with sort-means pruning        (Section 2.2 item 3, Algorithm 2;
 *                 stopping test of Section 3.3)
 *   kq_map        nearest palette colour per pixel, and SSE     (Section 1; MSE of Section 3.1, Eq. 2)
 *
 * Conventions for every entry point:
 *  - Pointers are DEVICE pointers unless the name starts with h_.  The caller
 *    allocates and owns every buffer, including the workspace `ws`; no entry
 *    point allocates device memory.
 *  - Every call is asynchronous on `stream` (a cudaStream_t; NULL is the legacy
 *    default stream) and returns after enqueueing its kernels.
 *  - The return value is a kq_status.  Invalid arguments (a null pointer, K
 *    outside 1..256, a workspace that is too small, a misaligned workspace)
 *    return KQ_EINVAL synchronously and enqueue nothing.  A failed kernel
 *    launch returns KQ_ECUDA.
 *  - Conditions found on the device (more unique colours than `capacity`, a
 *    barrier wait that timed out) are written to a status word inside `ws`.
 *    kq_status_read() returns it.  The first error is kept until
 *    kq_status_clear().
 *  - Colours are 24-bit keys (R << 16) | (G << 8) | B.  Pixels are packed
 *    HWC RGB8, 3 bytes per pixel, in any alignment.
 *  - Ties between equally near centres or palette entries go to the lowest index.
 *  - The workspace must be zero-filled once (kq_workspace_init()) before its
 *    first use; the library keeps its table regions zeroed between calls.
 *    Calls that share one workspace must be ordered on the GPU (one stream,
 *    or events); calls on separate workspaces are independent.
 *  - K is at most 256, so a palette index fits in a uint8_t.
 */
#ifndef KQ_H
#define KQ_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define KQ_API __attribute__((visibility("default")))
#else
#define KQ_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st *kq_stream_t; /* the same type as cudaStream_t */

typedef enum {
    KQ_OK = 0,
    KQ_EINVAL = -1,    /* invalid argument (synchronous) */
    KQ_ECAPACITY = -2, /* more unique colours than the caller's capacity (device status) */
    KQ_ECUDA = -3,     /* a CUDA runtime call failed */
    KQ_ETIMEOUT = -4,  /* a device-side wait passed its time limit (device status) */
    KQ_ENOMEM = -5     /* the workspace is too small for the request */
} kq_status;

/* Initialization schemes (Section 2.3).  KQ_INIT_USER: the caller's centres. */
typedef enum {
    KQ_INIT_FGY = 0, /* Forgy: K distinct unique colours, uniformly */
    KQ_INIT_LBG = 1, /* splitting (Linde-Buzo-Gray) from the centroid */
    KQ_INIT_MMX = 2, /* minmax (farthest first) */
    KQ_INIT_DEN = 3, /* density-based: 64 uniform cells, seats by pixel count */
    KQ_INIT_VAR = 4, /* maximum variance: medians of K groups on the widest channel */
    KQ_INIT_SFF = 5, /* subset farthest first on ceil(2 K ln K) random colours */
    KQ_INIT_KPP = 6, /* k-means++ (D^2 sampling, pixel-weighted) */
    KQ_INIT_USER = 7,
    KQ_INIT_WU = 8   /* Wu's greedy orthogonal bipartitioning (Section 3.3; the WSM-WU initializer):
                        32^3 cells, the box of largest weighted variance split by the cut minimizing
                        the sum of the halves' variances, centres = box means */
} kq_init;

/* Parameters the paper leaves open; pass NULL for the defaults in brackets. */
typedef struct kq_seed_params {
    double lbg_eps;    /* LBG perturbation per channel, 0-255 units [1.0] */
    double conv_eps;   /* LBG refinement: relative SSE threshold [1e-4] */
    int32_t max_iter;  /* LBG refinement: iteration limit [100] */
    int32_t reserved;  /* must be 0 */
} kq_seed_params;

/* Device-side statistics written by kq_lloyd (caller-owned device memory). */
typedef struct kq_lloyd_stats {
    int32_t iters;     /* assignment+update passes run */
    int32_t converged; /* 1 when the relative SSE test of Section 3.3 fired */
    int32_t k_eff;     /* min(K, N') */
    int32_t status;    /* KQ_OK, or the device error that stopped the run */
    int64_t ndc;       /* distance calculations, the paper's NDC count, summed over iterations */
    double sse;        /* pixel-weighted SSE of the last assignment (Eq. 1) */
    double sse_prev;   /* SSE of the assignment before it (0 after one pass) */
} kq_lloyd_stats;

/* kq_lloyd flags */
#define KQ_LLOYD_LABELS_IN 1u /* `labels` holds a previous assignment: prune from the first pass */
#define KQ_LLOYD_DENSE 2u     /* full search of all K centres in every pass (no pruning) */

/*
 * Bytes of workspace needed for images of up to `max_pixels` pixels and
 * palettes of up to `max_K` colours (1..256).  Returns 0 for invalid sizes.
 * The workspace must be 256-byte aligned (any cudaMalloc/torch allocation is).
 */
KQ_API size_t kq_workspace_size(int64_t max_pixels, int32_t max_K);

/* Zero-fills the workspace on `stream` (once, before its first use). */
KQ_API int kq_workspace_init(void *ws, size_t ws_bytes, kq_stream_t stream);

/*
 * Unique colours and their pixel counts (Section 2.2: sampling of the pixels
 * with unique colours, each weighted by its frequency -- a colour histogram).
 *   rgb        n_pixels x 3 bytes, packed HWC.
 *   keys       out: N' unique colours in ascending key order (capacity entries).
 *   weights    out: pixel count of each unique colour (integer; the paper's
 *              weights are these divided by n_pixels).
 *   capacity   entries available in keys and weights.
 *   n_unique   out (device int32): min(N', capacity).  When N' > capacity the
 *              first `capacity` colours are written and the device status
 *              becomes KQ_ECAPACITY.
 * n_pixels may be 0 (then N' = 0).  Bit-exact: the result is unique.
 */
KQ_API int kq_histogram(const uint8_t *rgb, int64_t n_pixels, uint32_t *keys, uint32_t *weights, int32_t capacity,
                 int32_t *n_unique, void *ws, size_t ws_bytes, kq_stream_t stream);

/*
 * kq_histogram over a deterministic subsample: only the pixels (x, y) with x and y
 * multiples of `stride`.  stride = 2 is the 2:1 subsampling in both directions of
 * Section 2.2 (data sampling), combined there with the unique-colour sampling;
 * stride = 1 is the whole image.
 *   rgb        height rows of width x 3 bytes; row y starts at rgb + y * pitch.
 *   pitch      bytes between rows, >= 3 * width.
 * Other arguments and results as kq_histogram.
 */
KQ_API int kq_histogram_strided(const uint8_t *rgb, int32_t height, int32_t width, int64_t pitch, int32_t stride,
                                uint32_t *keys, uint32_t *weights, int32_t capacity, int32_t *n_unique, void *ws,
                                size_t ws_bytes, kq_stream_t stream);

/*
 * Initial centres by a generic scheme of Section 2.3.
 *   keys, weights, n_unique   the output of kq_histogram.
 *   K          palette size, 1..256.  When K >= N' the centres are the N'
 *              unique colours in key order, padded with copies of the last.
 *   scheme     a kq_init value other than KQ_INIT_USER.
 *   seed       random seed.  Draw number i of stream s is output
 *              s * 2^32 + i + 1 of SplitMix64 seeded with `seed`; an integer
 *              in [0, m) is the high 64 bits of that output times m.
 *   params     NULL for the defaults (LBG only).
 *   centers    out: K x 3 doubles (FP64; integer-valued except for LBG).
 * Every scheme except LBG is bit-exact (integer arithmetic throughout).
 */
KQ_API int kq_seed(const uint32_t *keys, const uint32_t *weights, const int32_t *n_unique, int32_t K, int32_t scheme,
            uint64_t seed, const kq_seed_params *params, double *centers, void *ws, size_t ws_bytes,
            kq_stream_t stream);

/*
 * Weighted Sort-Means (Algorithm 2): repeated passes of
 *   assignment -- nearest centre per unique colour, scanning the centres in
 *                 increasing distance from the previous centre p and stopping
 *                 once d(c_p, c_t) rules out any nearer centre (Section 2.2,
 *                 item 3); distances in FP32; the labels equal those of a full
 *                 FP32 search (lowest index on ties);
 *   update     -- weighted means from exact int64 sums, divided in FP64; an
 *                 empty cluster keeps its centre;
 *   stop test  -- after pass i, stop when SSE_i == 0 or, for i > 1,
 *                 (SSE_{i-1} - SSE_i) / SSE_i <= eps (Section 3.3); eps < 0
 *                 runs exactly max_iter passes (the protocol of Section 3.2).
 *   centers    in: K x 3 FP64 seeds; out: the final centres.
 *   max_iter   pass limit, >= 1.
 *   flags      KQ_LLOYD_LABELS_IN, KQ_LLOYD_DENSE.
 *   labels     N' bytes: in (with KQ_LLOYD_LABELS_IN) and out (last assignment).
 *   palette    out: K x 3 bytes, each centre rounded half-up: floor((2S+W)/(2W))
 *              per channel from the exact sums; an empty cluster rounds its
 *              held centre (floor(c + 0.5), clamped to 0..255).
 *   stats      out (device): see kq_lloyd_stats.  May be NULL.
 *   sse_hist   out (device, nullable): SSE of each pass, max_iter doubles.
 * The whole loop runs on the device as one cooperative launch; the host never
 * waits between passes.
 */
KQ_API int kq_lloyd(const uint32_t *keys, const uint32_t *weights, const int32_t *n_unique, int32_t K, double *centers,
             double eps, int32_t max_iter, uint32_t flags, uint8_t *labels, uint8_t *palette, kq_lloyd_stats *stats,
             double *sse_hist, void *ws, size_t ws_bytes, kq_stream_t stream);

/*
 * Pixel mapping (Section 1; Section 2.1 notes that k-means maps by a full
 * palette search): idx[i] = argmin_k |rgb_i - palette_k|^2 in exact integer
 * arithmetic, lowest index on ties.  The search per pixel is exact but visits
 * only the palette entries that can be nearest somewhere in the pixel's cell of
 * 8 x 8 x 8 colours (found from the palette alone at the start of the call).
 *   rgb        n_pixels x 3 bytes, packed HWC, any alignment.
 *   palette    K x 3 bytes (device).   idx   out: n_pixels bytes.
 *   sse_num    out (device int64, nullable): sum over the pixels of the squared
 *              error, the numerator of the MSE of Section 3.1 (Eq. 2).
 * Needs no histogram and keeps no state between calls.
 */
KQ_API int kq_map(const uint8_t *rgb, int64_t n_pixels, const uint8_t *palette, int32_t K, uint8_t *idx,
                  int64_t *sse_num, void *ws, size_t ws_bytes, kq_stream_t stream);

/* ------------------------------------------------------------------ batches
 * Many images of uneven size and K in one persistent launch (the paper treats
 * one image at a time; this runs its four steps for every image of a batch).
 * Each image is taken from start to finish -- histogram, seeding, Weighted
 * Sort-Means, mapping -- by one group of thread blocks: a thread-block cluster of
 * `cluster` CTAs for images of more than `split_pixels` pixels, one CTA for the
 * others.  Groups pull images from a device-side queue in the order of
 * kq_batch_plan (largest estimated work first).  Per image the results are those
 * of kq_histogram, kq_seed, kq_lloyd and kq_map on the same inputs, except that
 * the FP32 SSE partials are summed over a different partition of blocks (the
 * stop test can therefore differ only when (SSE_{i-1} - SSE_i) / SSE_i lies within
 * about 1e-6 relative of eps).
 */

/* Per-image results, written by kq_batch_run (device memory, caller-owned). */
typedef struct kq_batch_result {
    int32_t status;       /* KQ_OK, KQ_EINVAL (bad item) or KQ_ECAPACITY (N' > capacity) */
    int32_t n_unique;     /* N' (also when above capacity) */
    kq_lloyd_stats lloyd; /* the final Lloyd run, as kq_lloyd writes it */
    int64_t sse_num;      /* sum over pixels of |pixel - palette[idx]|^2 (MSE numerator, Eq. 2) */
    int64_t t_ns[5];      /* device clock (%globaltimer, ns) when the image's group started it and
                             finished its histogram, seeding, Lloyd and mapping steps */
} kq_batch_result;

/* One image of a batch.  Host and device use the same layout: the array passed
 * to kq_batch_run is a device copy of the host array given to kq_batch_plan.
 * All pointers are device pointers owned by the caller. */
typedef struct kq_batch_item {
    const uint8_t *rgb;       /* n_pixels x 3 bytes, packed RGB8, any alignment */
    uint8_t *idx;             /* out: n_pixels palette indices */
    uint32_t *keys;           /* out: capacity entries, unique colours ascending (16-byte aligned) */
    uint32_t *weights;        /* out: capacity entries, pixel counts (16-byte aligned) */
    uint8_t *labels;          /* out: capacity entries, last assignment */
    void *scratch;            /* kq_batch_scratch_bytes(capacity) bytes, 256-byte aligned */
    double *centers;          /* K x 3; in for KQ_INIT_USER, out: final centres */
    uint8_t *palette;         /* out: K x 3 bytes (rounding as kq_lloyd) */
    kq_batch_result *result;  /* out */
    int64_t n_pixels;         /* >= 0 */
    uint64_t seed;            /* random stream seed of the scheme */
    double eps;               /* stop test of kq_lloyd */
    double lbg_eps;           /* KQ_INIT_LBG: split perturbation (kq_seed_params.lbg_eps) */
    double lbg_conv_eps;      /* KQ_INIT_LBG: refinement threshold */
    int32_t lbg_max_iter;     /* KQ_INIT_LBG: refinement pass limit (>= 1 for LBG) */
    int32_t K;                /* 1..256 */
    int32_t scheme;           /* kq_init */
    int32_t max_iter;         /* >= 1 */
    int32_t capacity;         /* length of keys / weights / labels; min(n_pixels, 2^24) always suffices */
    int32_t reserved;         /* 0 */
} kq_batch_item;

/* Launch shape: cluster size (1, 2, 4, 8 or 16; 1 = single CTAs only) and the
 * pixel count above which an image goes to a cluster. */
typedef struct kq_batch_config {
    int32_t cluster;
    int32_t reserved;
    int64_t split_pixels;
} kq_batch_config;

/* Bytes of kq_batch_item.scratch for `capacity` unique colours (D^2 and the
 * k-means++ step sums). */
KQ_API size_t kq_batch_scratch_bytes(int32_t capacity);

/* Workspace bytes of kq_batch_run on the current device: one slot of about
 * 69 MiB (counter table, bitmaps, seeding and Lloyd scratch) per resident CTA.
 * Zero-fill it once before first use (the library keeps its tables zeroed). */
KQ_API size_t kq_batch_workspace_size(void);

/* Largest cluster size kq_batch_run can launch on the current device (>= 1). */
KQ_API int32_t kq_batch_max_cluster(void);

/* Host-side planner: validates h_items (KQ_EINVAL on a bad item) and writes the
 * processing order to h_order (n_items entries): first the images above
 * cfg->split_pixels (when cfg->cluster > 1), then the rest, each class in
 * decreasing n_pixels * (1 + K / 12).  *h_n_big = size of the first class. */
KQ_API int kq_batch_plan(const kq_batch_item *h_items, int32_t n_items, const kq_batch_config *cfg, int32_t *h_order,
                         int32_t *h_n_big);

/* Runs the whole batch: one memset of the queue counters and one launch,
 * asynchronous on `stream` (capturable in a CUDA graph).  `order` is a device copy
 * of kq_batch_plan's order, n_big its class split.  Per-image errors go to the
 * item's result; argument errors return KQ_EINVAL, a workspace smaller than
 * kq_batch_workspace_size() for this cluster size KQ_ENOMEM.  The workspace
 * must not be shared with a concurrent call. */
KQ_API int kq_batch_run(const kq_batch_item *items, int32_t n_items, const int32_t *order, int32_t n_big,
                        const kq_batch_config *cfg, void *ws, size_t ws_bytes, kq_stream_t stream);

/* Autotuner: times kq_batch_run on this batch for each launch shape the device
 * supports (single CTAs; clusters of 2..16 with split_pixels 2^18, 2^20, 2^22),
 * keeps the fastest (best of two timed runs after a warm-up), writes its order
 * to `order` (device) and returns the shape, its n_big and its time (ms).
 * Synchronizes `stream`; the items' outputs hold the last timed run. */
KQ_API int kq_batch_tune(const kq_batch_item *h_items, const kq_batch_item *items, int32_t n_items, int32_t *order,
                         kq_batch_config *h_best, int32_t *h_n_big, float *h_best_ms, void *ws, size_t ws_bytes,
                         kq_stream_t stream);

/*
 * Live batches: images join a launch that is already running.  (The paper treats
 * one image at a time; this is the serving form of the batched launch above.)
 * A queue in page-locked host memory (cudaHostAlloc, or a pinned tensor), which
 * the host and the running kernel both read and write, holds two rings of items,
 * one per class: class 0 is taken by thread-block clusters of cfg->cluster CTAs,
 * class 1 by single CTAs (a launch with cluster = 1 serves class 1 only).  The
 * host publishes an item with kq_live_publish; a group of the running launch
 * claims it, runs the four steps exactly as kq_batch_run would, and marks it done;
 * kq_live_done reads the mark.  Per image the results are those of kq_batch_run.
 *
 * Memory: every pointer of a live item must be reachable by the running kernel
 * while it runs.  The item's input pixels must be written by the host thread that
 * publishes it (or be ordered before the publication by that thread, e.g. by
 * waiting for a copy's completion), and must not change until the item is done;
 * its outputs may be read once kq_live_done returns 1.  Buffers of a finished item
 * may be reused for a later one.
 *
 * A live launch exits when the queue is closed and both rings are drained, or after
 * `idle_us` microseconds without an item to take (a bounded wait: nothing spins
 * without limit); items published later wait for the next kq_live_run, which
 * continues from the claim counters in `ws`.  Only one live launch may run on a
 * queue and its workspace at a time, and no kq_batch_run may share the workspace.
 */
typedef struct kq_live_queue {
    uint32_t tail[2];       /* items published per class (written by kq_live_publish) */
    uint32_t closed;        /* 1 after kq_live_close */
    uint32_t capacity;      /* ring slots per class */
    uint32_t reserved[12];
    /* followed by kq_batch_item items[2][capacity] and uint32_t done[2][capacity] */
} kq_live_queue;

/* Bytes of a live queue with `capacity` ring slots per class (0 for capacity < 1). */
KQ_API size_t kq_live_bytes(int32_t capacity);

/* Host: empties the queue at `q` (kq_live_bytes(capacity) bytes of page-locked
 * host memory). */
KQ_API int kq_live_init(kq_live_queue *q, int32_t capacity);

/* Zeroes the claim counters of a live queue in the batch workspace `ws` (asynchronous
 * on `stream`); call it once for a freshly initialised queue, before its first
 * kq_live_run. */
KQ_API int kq_live_reset(void *ws, size_t ws_bytes, kq_stream_t stream);

/* Host: publishes a copy of *item (host memory) in class `cls` and returns its
 * sequence number in *h_seq.  KQ_ECAPACITY when the ring slot it needs still holds
 * an item that is not done; KQ_EINVAL for an invalid item, as kq_batch_plan checks
 * them, or after kq_live_close.  One host thread publishes at a time (the tail is
 * read and then advanced without a lock). */
KQ_API int kq_live_publish(kq_live_queue *q, int32_t cls, const kq_batch_item *item, int64_t *h_seq);

/* Host: 1 when item `seq` of class `cls` is done (its outputs are written), else 0.
 * The mark lives in the item's ring slot: once a later item is published into the
 * same slot (which kq_live_publish allows only after this one is done), the call
 * answers for that item instead, so read it before publishing `capacity` more items
 * of the class. */
KQ_API int kq_live_done(const kq_live_queue *q, int32_t cls, int64_t seq);

/* Host: no more items will be published; the running launch exits once drained. */
KQ_API int kq_live_close(kq_live_queue *q);

/* Launches the persistent live kernel on `stream` (asynchronous): cfg->cluster
 * CTAs per group for class 0 (cfg->split_pixels is not used: the publisher picks
 * the class), idle limit `idle_us` (>= 1).  KQ_EINVAL when `q` is not page-locked
 * host memory the device can reach; KQ_ENOMEM when `ws` is smaller than
 * kq_batch_workspace_size(). */
KQ_API int kq_live_run(kq_live_queue *q, const kq_batch_config *cfg, uint32_t idle_us, void *ws, size_t ws_bytes,
                       kq_stream_t stream);

/*
 * kq_lloyd without a workspace (the paper has no counterpart: this entry point
 * exists for callers of this library that cannot allocate device memory -- for
 * example a plug-in inside a host application that owns the whole device memory
 * budget and hands the plug-in only its input and output buffers, or code that
 * must not trigger the device-wide synchronisation of cudaMalloc/cudaFree).
 *
 * Same arguments, results and device-side behaviour as kq_lloyd, minus `ws`.
 * Its scratch (control block, cluster sums, SSE partials and the sorted
 * centre-distance rows) is one static device array of 356,352 bytes inside
 * libkq.so; every GPU that loads the library holds it
 * until the process exits.
 *  - Limit: K <= 256 (the array holds sums and rows for 256 centres); K > 256,
 *    like any invalid argument, returns KQ_EINVAL.
 *  - It allocates nothing: no cudaMalloc, no cudaFree, no allocating library call.
 *  - Every call looks up the array's device address in the current context
 *    (cudaGetSymbolAddress, a host-side query); on a device that has not run
 *    the library before, that first lookup loads its module, so make the first
 *    call on each device before any stream capture.
 *  - Every call clears the control block (status, barrier counters) and uses
 *    the same array: calls that overlap on the GPU (several streams, several
 *    host threads on one device) race and give wrong results.  Order them.
 *  - Device-side errors go to stats->status (the array's status word is not
 *    readable through kq_status_read).
 */
KQ_API int kq_lloyd_noalloc(const uint32_t *keys, const uint32_t *weights, const int32_t *n_unique, int32_t K,
                            double *centers, double eps, int32_t max_iter, uint32_t flags, uint8_t *labels,
                            uint8_t *palette, kq_lloyd_stats *stats, double *sse_hist, kq_stream_t stream);

/*
 * The plain k-means baseline of Table 1 (Section 3.2): every pixel as its own
 * point.  Writes keys[i] = (R << 16) | (G << 8) | B of pixel i (in pixel order,
 * not unique), weights[i] = 1 when `weights` is not NULL, and *n_out = n_pixels
 * when `n_out` is not NULL, so that kq_lloyd run on (keys, weights, n_out) with
 * KQ_LLOYD_DENSE is k-means on all N pixels.  Not a step of Weighted Sort-Means.
 *   rgb        n_pixels x 3 bytes.   keys, weights   n_pixels entries (device).
 * Returns KQ_EINVAL for n_pixels outside 0 .. 2^31 - 1 or a missing buffer.
 */
KQ_API int kq_pixel_keys(const uint8_t *rgb, int64_t n_pixels, uint32_t *keys, uint32_t *weights, int32_t *n_out,
                         kq_stream_t stream);

/*
 * Failure detection.  Every device-side wait of the kernels that use `ws` (the
 * grid barriers of kq_lloyd and of the whole-grid seeding, the exchanges of the
 * cluster seeding) gives up after a time limit: it writes KQ_ETIMEOUT to the
 * status word (and to kq_lloyd's stats), the other waiters follow, and the
 * kernel returns, leaving the context usable.  This call sets, for the launches
 * enqueued after it on `ws`:
 *   wait_limit_us      the limit in microseconds (0: the default of 4 s);
 *   missing_arrivals   arrivals every such wait expects beyond the blocks that
 *                      take part -- 0 in normal use; a positive value makes the
 *                      waits run out, which is how the timeout path is tested
 *                      without faulting or hanging the GPU.
 * Asynchronous on `stream`.  kq_status_clear() resets both to 0.
 */
KQ_API int kq_set_wait_limit(void *ws, size_t ws_bytes, uint32_t wait_limit_us, uint32_t missing_arrivals,
                             kq_stream_t stream);

/* Distance calculations of the last kq_map on `ws` (the paper's NDC for the
 * mapping step: palette entries examined, summed over the pixels), copied to
 * *h_ndc (synchronizes `stream`). */
KQ_API int kq_map_ndc_read(const void *ws, int64_t *h_ndc, kq_stream_t stream);

/* ------------------------------------------------------------------ CIE L*a*b*
 * k-means in the CIE L*a*b* colour space (Section 2.1 names L*a*b* beside RGB as a
 * space k-means runs in): the unique colours of kq_histogram become L*a*b* points,
 * Weighted Sort-Means runs on them (the same pruning, update and stop test as
 * kq_lloyd), and each pixel takes the label of its colour.
 *
 * A point is one uint64_t: bits 0-15, 16-31 and 32-47 hold L*, a* and b* times 256,
 * rounded to nearest (ties to even), as two's-complement 16-bit integers (every
 * sRGB colour's L*a*b* lies within +-128); bits 48-63 are zero.  Centres are given
 * in the same units (L*a*b* x 256) as FP64.
 */

/* L*a*b* point of each unique colour: 8-bit sRGB (IEC 61966-2-1) made linear, the
 * sRGB matrix to CIE XYZ (D65), CIE 1976 L*a*b* relative to the D65 white
 * (X_n = 0.95047, Y_n = 1, Z_n = 1.08883), all in FP64 with every operation
 * rounded separately.  points: N' entries (device).  Asynchronous. */
KQ_API int kq_lab_points(const uint32_t *keys, const int32_t *n_unique, uint64_t *points, kq_stream_t stream);

/* Initial centres among the points (Section 2.3).  scheme: KQ_INIT_FGY only (K
 * distinct points with the draws of kq_seed's Forgy; K >= N' gives the points in
 * order, padded with the last).  centers: K x 3 FP64 in point units. */
KQ_API int kq_seed_points(const uint64_t *points, const int32_t *n_unique, int32_t K, int32_t scheme, uint64_t seed,
                          double *centers, kq_stream_t stream);

/* Weighted Sort-Means on the points: kq_lloyd with the points' three coordinates in
 * place of a colour's three bytes (exact int64 sums of weight x coordinate, FP64
 * division, FP32 distances, the same pruning, ties and stop test).  No palette:
 * kq_lab_palette turns the centres into sRGB colours. */
KQ_API int kq_lloyd_points(const uint64_t *points, const uint32_t *weights, const int32_t *n_unique, int32_t K,
                           double *centers, double eps, int32_t max_iter, uint32_t flags, uint8_t *labels,
                           kq_lloyd_stats *stats, double *sse_hist, void *ws, size_t ws_bytes, kq_stream_t stream);

/* sRGB palette of K centres in point units: the inverse of kq_lab_points (L*a*b* to
 * XYZ to linear RGB by the inverse sRGB matrix, companding), each channel clamped
 * to [0, 1] and rounded half up to 0..255, in FP64. */
KQ_API int kq_lab_palette(const double *centers, int32_t K, uint8_t *palette, kq_stream_t stream);

/* Mapping in L*a*b* (or any space Lloyd ran in over the unique colours): each
 * pixel's index is the label of its colour in (keys, labels), as kq_histogram and
 * kq_lloyd_points left them.  A pixel whose colour is not among `keys` gets 0 and
 * sets KQ_EINVAL in the device status word.  Uses the workspace's colour table,
 * which is zero again when the call's kernels finish. */
KQ_API int kq_map_labels(const uint8_t *rgb, int64_t n_pixels, const uint32_t *keys, const int32_t *n_unique,
                         const uint8_t *labels, uint8_t *idx, void *ws, size_t ws_bytes, kq_stream_t stream);

/* Device status word of `ws` copied to *h_status (synchronizes `stream`). */
KQ_API int kq_status_read(const void *ws, int32_t *h_status, kq_stream_t stream);

/* Resets the device status word of `ws` to KQ_OK, with the abort flag and the
 * settings of kq_set_wait_limit (asynchronous). */
KQ_API int kq_status_clear(void *ws, kq_stream_t stream);

/* Static description of a status code. */
KQ_API const char *kq_strerror(int status);

#ifdef __cplusplus
}
#endif

#endif /* KQ_H */
