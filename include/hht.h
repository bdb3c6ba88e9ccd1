/*
 * hht.h - C ABI of the GB300 hierarchical Hough transform library (libhht.so).
 *
 * The library runs the hierarchical Hough transform for straight lines of
 * Singh & Bhatia, "A Fast Decision Technique for Hierarchical Hough Transform
 * for Line Detection" (arXiv:1007.0547), on one CUDA device:
 *
 *   - Each edge point (x, y) is the line b = y - m*x of the (m, b) parameter
 *     space (Section 1, slope-intercept form).  Points are processed in two
 *     halves: half 0 ("ALPHA") as given, half 1 ("BETA") with x and y swapped,
 *     so that both halves only need slopes |m| <= 1 (Section 3).  Every point
 *     enters both halves.
 *   - The parameter space m in [-1, 1], b in [-2L, 2L], L the smallest power
 *     of two >= max(W, H), is the level-0 region.  A region is split into the
 *     quadrants NE, NW, SW, SE (Section 3).
 *   - A line's 4-bit code for a region has one bit per corner in the order NE,
 *     NW, SW, SE; a bit is 1 when that corner lies strictly below the line
 *     (Section 2: F = y0 - m*x0 - b < 0; a corner on the line counts as above).
 *     The line votes for the region when the code is neither 0000 nor 1111
 *     (Section 3).
 *   - A region whose votes reach T (votes >= T) is split again; the level-0
 *     region is always split.  At level `depth` the regions are cells of a
 *     K x K grid, K = 2^depth, and each cell that reaches T is reported as a
 *     leaf (Section 3: the paper's solution() output, without
 *     the removal of plotted voters).
 *
 * Leaf cell (i, j) of half h spans m in [-1 + 2i/K, -1 + 2(i+1)/K] and
 * b in [-2L + 4Lj/K, -2L + 4L(j+1)/K] (in the half's own coordinates).
 * Every decision is an exact integer comparison, so results are unique.
 * Leaves are reported half 0 first, each half in the order in which the
 * paper's depth-first traversal reaches them (children quad1..quad4 = NE, NW,
 * SW, SE at every level), i.e. the order of its solution() calls.
 *
 * Errors: every call returns HHT_OK (0) or a negative HHT_E_* code.  No call
 * aborts, asserts or traps; argument errors are found before any device work.
 * Threads: a context is used by one host thread at a time.
 */
#ifndef HHT_H_
#define HHT_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/*
 * Size limits.  Images are at most HHT_MAX_SIDE pixels on a side and
 * HHT_MAX_DEPTH levels deep.  One level of a job holds at most 2^32 - 2
 * regions (HHT_E_NOMEM beyond).  The voters that a level's regions hand on
 * to their children are summed in 64 bits at every stage of the selection,
 * so a level's voter streams have no 32-bit limit; their size is bounded by
 * device memory (HHT_E_NOMEM when a single image's level does not fit).
 */
#define HHT_MAX_DEPTH 24
#define HHT_MAX_SIDE 32767

enum {
    HHT_OK = 0,
    HHT_E_ARG = -1,          /* bad argument: NULL, n < 0, W/H outside [1, 32767],
                                depth outside [1, 24], T < 1, bad image count */
    HHT_E_RANGE = -2,        /* a point lies outside [0, W) x [0, H); result invalid */
    HHT_E_CAPACITY = -3,     /* leaf buffer too small; n_leaves holds the needed count */
    HHT_E_NOMEM = -4,        /* device memory (or the context's budget) exhausted, or one level of a job
                                could hold more than 2^32 - 2 regions (4 children per parent) */
    HHT_E_TIMEOUT = -5,      /* a bounded device-side wait expired; result invalid */
    HHT_E_CUDA = -6,         /* a CUDA runtime call failed */
    HHT_E_PENDING = -7,      /* hht_poll: the request has not finished yet */
    HHT_E_UNKNOWN_TICKET = -8
};

/* Edge point of an image, 0 <= x < W, 0 <= y < H. */
typedef struct {
    int16_t x, y;
} hht_point;

/* One reported cell: half (0 = as given, 1 = x/y swapped), cell indices (i, j)
 * on the K x K grid of the half, and its vote count (>= T). */
typedef struct {
    uint32_t half, i, j, votes;
} hht_leaf;

/* Per half and level: regions tested, regions passed (votes >= T; the
 * level-0 region always counts as passed), votes summed over the tested
 * regions, and 4-bit codes evaluated (n at level 0, four per voter of every
 * passed parent below). */
typedef struct {
    uint64_t tested, passed, votes, tests;
} hht_level_stats;

/* Result of one image.  The caller owns `leaves` (host or device memory of
 * the context's device, leaf_capacity entries); the library fills the rest. */
typedef struct {
    hht_leaf *leaves;
    uint64_t leaf_capacity;
    uint64_t n_leaves;                               /* out: leaves found */
    int32_t depth, L;                                /* out: grid depth, frame side */
    int32_t status;                                  /* out: HHT_OK or HHT_E_* of this image */
    int32_t reserved;
    hht_level_stats stats[2][HHT_MAX_DEPTH + 1];     /* out: [half][level], levels 0..depth */
} hht_result;

/* One image of a batch or a serving request.  `points` is host memory or
 * device memory of the context's device (n entries, read only). */
typedef struct {
    const hht_point *points;
    int64_t n;
    int32_t W, H, depth, T;
} hht_image;

typedef struct hht_ctx hht_ctx;

/*
 * Create a context on CUDA device `device`, issuing all work on `cuda_stream`
 * (a cudaStream_t; NULL means the legacy default stream).
 * mem_budget_bytes caps the device scratch memory the context may hold
 * (0 = no cap beyond the device's free memory).  The context owns that
 * scratch memory; it is freed by hht_destroy().
 * Errors: HHT_E_ARG (out == NULL, bad device), HHT_E_CUDA.
 */
int hht_create(hht_ctx **out, int device, void *cuda_stream, uint64_t mem_budget_bytes);

/*
 * A caller's device allocator, for processes whose device memory belongs to
 * another allocator (for instance PyTorch's caching allocator): alloc returns
 * at least `bytes` of device memory of the context's device, 256-byte aligned
 * (NULL when it cannot), for use on `cuda_stream`; free takes back a block
 * with the size it was asked for.  Both are called only from inside hht_*
 * calls on the context, on the calling thread; a block is freed only after
 * the context's stream has finished with it.
 */
typedef struct {
    void *(*alloc)(size_t bytes, void *cuda_stream, void *user);
    void (*free)(void *ptr, size_t bytes, void *cuda_stream, void *user);
    void *user;
} hht_allocator;

/*
 * hht_create with every device allocation of the context (its scratch
 * memory) made through `allocator` (NULL: cudaMalloc and cudaFree, as
 * hht_create).  The budget still caps what the context holds.
 * Errors: as hht_create, and HHT_E_ARG when alloc or free is NULL.
 */
int hht_create_with_allocator(hht_ctx **out, int device, void *cuda_stream, uint64_t mem_budget_bytes,
                              const hht_allocator *allocator);

/* Destroy a context (NULL is ignored).  Waits for the context's stream. */
void hht_destroy(hht_ctx *ctx);

/*
 * Detect lines in one image (Section 3, both halves).  `points` holds n edge
 * points in host memory or in device memory of the context's device; n = 0 is
 * valid.  On return the work is complete (the call synchronises the stream):
 * out->leaves[0 .. n_leaves) hold the leaves in depth-first order (see above)
 * and out->stats[h][l] the statistics for levels 0..depth.
 * Errors: HHT_E_ARG (checked before any device work), HHT_E_RANGE (a point
 * outside the image), HHT_E_CAPACITY (out->n_leaves = required count; fetch
 * them with hht_fetch_leaves), HHT_E_NOMEM, HHT_E_TIMEOUT, HHT_E_CUDA.
 */
int hht_detect(hht_ctx *ctx, const hht_point *points, int64_t n, int32_t W, int32_t H, int32_t depth,
               int32_t T, hht_result *out);

/*
 * Detect lines in `count` independent images in one batched pass: all images
 * and both halves of each advance level by level through the same kernel
 * launches (see hht_set_batch_mode for the one-launch form).  outs[k] receives
 * image k's result exactly as hht_detect would produce it.  Returns HHT_OK
 * when every image succeeded, else the first failing image's code (each
 * outs[k].status holds that image's own code).
 */
int hht_detect_batch(hht_ctx *ctx, const hht_image *images, int32_t count, hht_result *outs);

/*
 * Copy the leaves of image `index` (0 for hht_detect) of the last
 * hht_detect / hht_detect_batch call on this context into `leaves` (host or
 * device memory, `capacity` entries), without running anything again.  This
 * completes the two-call protocol: after HHT_E_CAPACITY the caller allocates
 * n_leaves entries and fetches them.  Valid until the next call that runs a
 * detection on the context.  Errors: HHT_E_ARG (no such image, NULL buffer),
 * HHT_E_CAPACITY (buffer smaller than the image's leaf count; nothing copied),
 * HHT_E_CUDA.
 */
int hht_fetch_leaves(hht_ctx *ctx, int32_t index, hht_leaf *leaves, uint64_t capacity);

/*
 * Copy all leaves of the last job (every image of the last hht_detect_batch)
 * with one copy: `leaves` receives *total entries (host or device memory,
 * `capacity` entries), and image k's leaves are leaves[offsets[k] ..
 * offsets[k] + counts[k]) (offsets and counts: one entry per image of the
 * job, may be NULL).  The job is the last hht_detect_batch call that passed
 * its argument checks: a call that returned HHT_E_ARG (or had count 0) did not
 * replace it, so size offsets and counts by that call's count.  Images that
 * failed have count 0.  With capacity < total nothing is copied (and offsets
 * and counts are not written) and HHT_E_CAPACITY is returned with *total set.
 * Errors: HHT_E_ARG, HHT_E_CAPACITY, HHT_E_CUDA.
 */
int hht_fetch_all_leaves(hht_ctx *ctx, hht_leaf *leaves, uint64_t capacity, uint64_t *offsets, uint64_t *counts,
                         uint64_t *total);

/*
 * Serving interface.  hht_submit() queues one request and returns at once;
 * its points (host or device memory) are copied, so the caller's buffer may
 * be reused when it returns.  hht_progress() runs one step of the engine's
 * level loop and returns when that step's kernels have finished, with the
 * number of requests in flight or waiting (or a negative error code: the
 * requests in flight then fail with it).  At each step waiting requests are
 * admitted in arrival order while 1024 request slots and the memory budget
 * allow.  The budget is the context's, capped at 85 % of the device memory
 * free at the first step (that 85 % when the context has none).  Admission
 * projects, for every step to come, the voter-list and region bounds of each
 * request in flight at the level it will then be at (at level l a line
 * votes in at most 2^l + (W - 1) 2^l / 2L + 2 cells; regions are at most 4^l
 * and the votes / T), and admits a request when the two voter-stream buffers
 * and the largest step's region buffers then need at most 90 % of the
 * budget; requests whose deep levels fall on different steps share it.  A
 * request that does not fit is passed over by later ones that do for at
 * most 12 steps, after which nothing is admitted until it fits.  A finished
 * request's leaves stay in device memory until it is polled.
 * hht_poll() returns HHT_E_PENDING until the request is done, then copies its
 * leaves into the caller's buffer (host or device memory; pinned host memory
 * is copied fastest), fills *out and releases the ticket; HHT_E_CAPACITY
 * (with out->n_leaves set) leaves the ticket valid for a larger buffer.  A
 * poll's copy runs on a stream of its own and does not wait for the step in
 * progress, so polls may come from other threads than hht_progress().
 */
int hht_submit(hht_ctx *ctx, const hht_image *image, uint64_t *ticket);
int hht_poll(hht_ctx *ctx, uint64_t ticket, hht_result *out);
int hht_progress(hht_ctx *ctx);

/*
 * Completion list of the serving interface: writes up to `capacity` tickets
 * of requests that have finished (successfully or not) and have not been
 * polled or listed before, oldest completion first, and their number into
 * *count, so that a client polls only finished requests.  Errors: HHT_E_ARG.
 */
int hht_done_tickets(hht_ctx *ctx, uint64_t *tickets, uint64_t capacity, uint64_t *count);

/*
 * Kernel timing.  hht_profile_enable(ctx, 1) resets the counters and makes the
 * context record CUDA events on its stream around every kernel it launches
 * (0 stops recording).  hht_profile_read() copies the accumulated counters.
 * "pass" is the per-level kernel that reads a voter stream once; its
 * algorithmic bytes are 8 per voter record read plus 8 per record written.
 * Errors: HHT_E_ARG (NULL).
 */
typedef struct {
    uint64_t launches;          /* kernels launched by the context */
    uint64_t pass_launches;
    uint64_t select_launches;
    uint64_t voters_read;       /* voter records read by pass launches */
    uint64_t voters_written;    /* voter records written by pass launches */
    uint64_t pass_bytes;        /* 8 * (voters_read + voters_written) */
    double pass_ms;             /* summed device time of the pass launches */
    double select_ms;
    double stage_ms;
    uint64_t graph_launches;   /* waves run as one CUDA-graph launch of the device-driven level loop */
    uint64_t graph_fallbacks;  /* graph launches that ran out of room and were rerun level by level */
    uint64_t edges_launches;        /* front-end (Sobel and split) launches */
    uint64_t edges_pixels;          /* pixels they read */
    uint64_t edges_points;          /* edge points they wrote */
    double edges_ms;                /* their summed device time */
    uint64_t graph_captures;        /* CUDA graphs of the level loop captured (the rest were replays) */
} hht_profile_counters;

int hht_profile_enable(hht_ctx *ctx, int on);
int hht_profile_read(hht_ctx *ctx, hht_profile_counters *out);

/*
 * Single-image detection that allocates no memory (no paper counterpart:
 * this is a library-integration variant of hht_detect).  For callers that
 * cannot let a library call cudaMalloc: processes whose device memory belongs
 * to another framework's allocator (a stray allocation can fail or fragment
 * its pool), and loops that cannot take the device-wide synchronisation of an
 * allocation or free.  All scratch lives in one static device array of
 * HHT_NOALLOC_SCRATCH_BYTES that every GPU loading the library holds until
 * the process exits; no context is needed.
 *   points: n points in host or device memory; leaves: caller buffer (host or
 *   device) of leaf_capacity entries; out: statistics, n_leaves and status
 *   (host); cuda_stream: the stream to run on (NULL = legacy default stream).
 * The call synchronises `cuda_stream` once per level (the level's totals size
 * the next level) and before it returns, on success and on every error after
 * its first device work.  The first call on a device looks up the array's
 * device address and keeps it for the process's life; a cudaDeviceReset
 * between calls is not supported.  The array keeps the previous call's contents; each call
 * clears what it needs.  Calls that overlap on the GPU (other streams or
 * threads on the same device) race on the array and must not be made.
 * Limits: n <= HHT_NOALLOC_MAX_POINTS, depth <= HHT_NOALLOC_MAX_DEPTH, at most
 * HHT_NOALLOC_MAX_LEAVES leaves, and the per-level voter lists must fit the
 * array; beyond them the call returns HHT_E_NOMEM (the limits on n and depth
 * are checked before any device work).
 * Errors: as hht_detect (HHT_E_CAPACITY leaves nothing to fetch: call again
 * with a larger buffer).
 */
#define HHT_NOALLOC_SCRATCH_BYTES (64u << 20)
#define HHT_NOALLOC_MAX_POINTS (1 << 20)
#define HHT_NOALLOC_MAX_DEPTH 16
#define HHT_NOALLOC_MAX_LEAVES (1 << 18)
int hht_detect_noalloc(const hht_point *points, int64_t n, int32_t W, int32_t H, int32_t depth, int32_t T,
                       hht_leaf *leaves, uint64_t leaf_capacity, hht_result *out, void *cuda_stream);

/*
 * Autotuning of the level kernel's tile shape: voters per warp chunk (one
 * segment reservation per child and chunk), threads per block and resident
 * blocks per SM; HHT_TUNE_SHAPES shapes are compiled, shape 0 is the default.
 * hht_autotune() runs `images` once per shape (plus one warm-up run), keeps
 * the shape whose level kernels took the least device time for this context,
 * stores it in *best and, if ms_per_shape is not NULL, the per-shape times
 * (HHT_TUNE_SHAPES doubles).  hht_set_tuning() selects a shape directly (for
 * instance one cached from an earlier hht_autotune).  Results never depend on
 * the shape.  Errors: HHT_E_ARG, and those of hht_detect_batch.
 */
#define HHT_TUNE_SHAPES 6
int hht_autotune(hht_ctx *ctx, const hht_image *images, int32_t count, int32_t *best, double *ms_per_shape);
int hht_set_tuning(hht_ctx *ctx, int32_t shape);

/*
 * Execution form of hht_detect and hht_detect_batch (the results are the same
 * in both).
 * HHT_BATCH_GRAPH (default): the device-driven level loop.  Every buffer is
 * sized from hard upper bounds of the job (a line crosses at most
 * 2^l + (W - 1) 2^l / (2L) + 2 regions of level l, and a region passes with T
 * votes or more), the stage kernel and every level's selection and level
 * kernel read their sizes from device memory, and the whole loop is one CUDA
 * graph, captured once per argument set and replayed: one graph launch and
 * one host synchronisation per job, first call included.  On the legacy
 * default stream (no capture possible) the same kernels are launched one after
 * another with no host synchronisation between them.  Jobs whose bounds do
 * not fit the memory budget, circle-test (FHT) jobs and subtree shards run in
 * the level form.
 * HHT_BATCH_LEVELS: one selection and one level-kernel launch per level, with
 * a host synchronisation per level and every buffer sized exactly from the
 * previous selection; a batch that does not fit the budget runs in waves.
 * HHT_BATCH_PERSISTENT is the earlier name of HHT_BATCH_GRAPH.
 * Errors: HHT_E_ARG.
 */
#define HHT_BATCH_LEVELS 0
#define HHT_BATCH_GRAPH 1
#define HHT_BATCH_PERSISTENT HHT_BATCH_GRAPH
int hht_set_batch_mode(hht_ctx *ctx, int32_t mode);

/*
 * Detection with the paper's solution() step (Section 3): the regions are
 * visited depth-first (quad1..quad4 = NE, NW, SW, SE), and when a cell of the
 * leaf level gets votes >= T its voters are plotted and removed from every
 * region visited after it, so each edge point is plotted at most once per
 * half.  Readings: removal is per half (ALPHA and BETA are two runs, and every
 * point enters both); the `tests` statistic counts the codes actually
 * evaluated (the voters of each tested region's parent that were not removed
 * by then).  out->leaves receives the accepted cells, half 0's then half 1's,
 * each in visiting order, with their votes when visited; `plotted` (NULL or
 * 2 * n bytes, host or device) receives one flag per point and half
 * (half-major).  The visiting order makes this a sequential walk: each
 * (image, half) is one block of four warps on the GPU, which share every
 * pass over a region's voters; hht_detect_removal_batch runs many
 * images at once (no plotted flags).  Every accepted cell plots at least T
 * points, so a buffer of 2 * (n / T + 1) leaves always suffices; with a
 * smaller one the call returns HHT_E_CAPACITY with n_leaves set and copies
 * nothing (these cells are not kept for hht_fetch_leaves: call again).
 * Errors: HHT_E_ARG, HHT_E_RANGE, HHT_E_CAPACITY, HHT_E_NOMEM, HHT_E_CUDA.
 */
int hht_detect_removal(hht_ctx *ctx, const hht_point *points, int64_t n, int32_t W, int32_t H, int32_t depth,
                       int32_t T, hht_result *out, uint8_t *plotted);
int hht_detect_removal_batch(hht_ctx *ctx, const hht_image *images, int32_t count, hht_result *outs);

/*
 * The edge points that solution() plotted (Section 3: the paper draws them on
 * the image), for image `index` of the context's last removal job
 * (hht_detect_removal: 0; hht_detect_removal_batch: the image's index), as a
 * W x H raster written on the device: row-major, one byte per pixel, bit 0
 * set where a point plotted in half 0 lies and bit 1 where one plotted in
 * half 1 lies, every other byte 0.  `raster` (host or device) holds
 * `capacity` >= W * H bytes.  Errors: HHT_E_ARG (NULL, no successful removal
 * job, index out of range, capacity below W * H), HHT_E_CUDA.
 */
int hht_removal_raster(hht_ctx *ctx, int32_t index, uint8_t *raster, uint64_t capacity);

/*
 * One shard of a detection split by subtrees (no paper counterpart: a way to
 * spread one large image over several GPUs).  Below level k = split_level the
 * regions of the two halves are independent given the points, so several
 * contexts (one per GPU) can each take some of the 2 * 4^k level-k regions:
 * every shard computes levels 0..k in full, and a level-k region (a, b) of
 * half h is split further only when keep[h * 4^k + a * 2^k + b] is non-zero
 * (keep: 2 * 4^k bytes in host or device memory).  Arguments and results are
 * those of hht_detect; the shard's leaves are those of its own subtrees, in
 * depth-first order.  The whole detection is the union of the shards'
 * leaves (merged in depth-first order) with statistics combined as: levels
 * below k from any one shard, at level k the `passed` counts summed and the
 * rest from any one shard, below k everything summed.  Every shard computes
 * levels 0..k, so k is best kept small.  Errors: as hht_detect, and HHT_E_ARG
 * for a NULL mask or split_level outside [1, min(depth, HHT_MAX_SPLIT_LEVEL)].
 */
#define HHT_MAX_SPLIT_LEVEL 10
int hht_detect_subtrees(hht_ctx *ctx, const hht_point *points, int64_t n, int32_t W, int32_t H, int32_t depth,
                        int32_t T, int32_t split_level, const uint8_t *keep, hht_result *out);

/*
 * Front end (Section 3): Sobel's gradient operator on a grey-level image and
 * the split of its edge points into ALPHA (points on lines of absolute slope
 * <= 1) and BETA (the rest), which the paper does while the gradient is
 * computed.  `image` holds W * H bytes, row-major (pixel (x, y) at
 * y * W + x), in host or device memory.  Readings of the paper:
 *   - Sobel's 3 x 3 responses gx (right column minus left, weights 1, 2, 1)
 *     and gy (row below minus row above) exist at interior pixels
 *     (1 <= x <= W-2, 1 <= y <= H-2); border pixels are never edge points;
 *   - a pixel is an edge point when gx^2 + gy^2 >= threshold^2;
 *   - the line through an edge point runs across its gradient (slope
 *     -gx / gy): ALPHA when |gx| <= |gy|, else BETA.
 * hht_edges() writes the two point lists (row-major order each) into the
 * caller's buffers (host or device) and their lengths into *n_alpha and
 * *n_beta; when a buffer is too small it copies nothing and returns
 * HHT_E_CAPACITY with the lengths set (call again with larger buffers).
 * hht_detect_image() runs the front end and then the detection of
 * hht_detect with ALPHA as half 0 and BETA (x and y swapped) as half 1,
 * instead of every point entering both halves: out->stats[0] and [1] are the
 * two halves' statistics, and the leaves are ALPHA's followed by BETA's
 * (hht_fetch_leaves index 0 after HHT_E_CAPACITY).
 * Errors: HHT_E_ARG (NULL, W or H outside [1, 32767], threshold < 0, depth or
 * T as for hht_detect), HHT_E_CAPACITY, HHT_E_NOMEM, HHT_E_TIMEOUT, HHT_E_CUDA.
 */
int hht_edges(hht_ctx *ctx, const uint8_t *image, int32_t W, int32_t H, int32_t threshold, hht_point *alpha,
              uint64_t alpha_capacity, uint64_t *n_alpha, hht_point *beta, uint64_t beta_capacity,
              uint64_t *n_beta);
int hht_detect_image(hht_ctx *ctx, const uint8_t *image, int32_t W, int32_t H, int32_t threshold, int32_t depth,
                     int32_t T, hht_result *out);

/*
 * Leaves -> lines (no paper counterpart: the paper stops at the peak cells;
 * this step is this library's own reading).  For image `index` of the last
 * job on the context (0 for hht_detect and hht_detect_image), leaves of the
 * same half whose cells touch (|di| <= 1 and |dj| <= 1) form one cluster, and
 * each cluster is one line, reported in the order of its first leaf in the
 * depth-first leaf order:
 *   - half, i, j, votes: its peak leaf (most votes; ties to the earlier leaf);
 *   - cells: leaves in the cluster; total_votes: V, their summed votes;
 *   - sum_i2 = sum of votes * (2i + 1), sum_j2 = sum of votes * (2j + 1): the
 *     exact vote-weighted centre m = (sum_i2 / V - K) / K,
 *     b = 2L (sum_j2 / V - K) / K (K = 2^depth, L the frame side).
 * A cell's own centre is m = (2i + 1 - K) / K, b = 2L (2j + 1 - K) / K.  Half 0
 * lines read y = m x + b; half 1 lines x = m y + b (x and y swapped back).
 * `lines` is host or device memory of `capacity` entries; *n_lines receives
 * the count.  With capacity < count nothing is copied and HHT_E_CAPACITY is
 * returned; the lines stay in the context, so a second call for the same
 * image (before the next detection) only copies them.  Errors: HHT_E_ARG
 * (NULL, no such image), HHT_E_CAPACITY, HHT_E_NOMEM, HHT_E_TIMEOUT,
 * HHT_E_CUDA.
 */
typedef struct {
    uint32_t half, i, j, votes;
    uint32_t cells, reserved;
    uint64_t total_votes, sum_i2, sum_j2;
} hht_line;
int hht_lines(hht_ctx *ctx, int32_t index, hht_line *lines, uint64_t capacity, uint64_t *n_lines);

/*
 * Membership test of hht_detect and hht_detect_batch on this context.
 * HHT_PREDICATE_EXACT (default): the paper's 4-bit corner code (Section 2).
 * HHT_PREDICATE_FHT: the circumscribed-circle test of the Fast Hough
 * Transform that the paper compares against (Sections 1 and 3; Table 1): a
 * line votes for a region when its distance from the region's centre is at
 * most the radius of the circle through the region's four corners.
 * Distances are taken in cell units, where every region is a square, and the
 * test G(centre)^2 <= 2 s^2 (x^2 + 4L^2) (s = region side in cells, G as in
 * the exact test) is decided exactly on integers.  Every line that crosses a
 * region also passes its circle, so FHT votes are a superset of the exact
 * ones (the paper's false votes).  The FHT form runs the same level loop, is
 * built for images with log2(L) + depth <= 27 (larger ones: HHT_E_ARG before
 * any device work) and is not used by the serving interface or the
 * persistent batch form (those always use the exact test).
 * Errors: HHT_E_ARG (NULL context, unknown predicate).
 */
#define HHT_PREDICATE_EXACT 0
#define HHT_PREDICATE_FHT 1
int hht_set_predicate(hht_ctx *ctx, int32_t predicate);

/*
 * Host-side fault injection, for tests of the failure path (no paper
 * counterpart).  HHT_FAULT_WITHHOLD_SCAN_TILE: in the next detection job
 * (hht_detect or hht_detect_batch) of this context, tile `arg` of every
 * selection launch's look-back scan (tiles of 1024 parent regions, in claim
 * order) publishes nothing.  The tiles after it then wait on a flag that
 * nothing sets; each wait gives up after its bounded spin (about a second or
 * two), the job returns HHT_E_TIMEOUT, and the context stays usable for the
 * next call.  A selection with at most `arg` + 1 tiles is unaffected.
 * HHT_FAULT_GRAPH_CAPACITY: in the next job of this context that runs in the
 * graph form, the kernels are told that the stream of level 1 holds at most
 * `arg` voter records (the buffer itself keeps its size), so that a level-1
 * stream longer than that makes the selection report an overflow, every later
 * kernel of the graph skips its work and the job is rerun level by level
 * (counted in graph_fallbacks).
 * HHT_FAULT_NONE clears a pending injection.  No GPU fault, trap or endless
 * wait is involved.  Errors: HHT_E_ARG (NULL context, unknown kind, arg
 * outside [0, 2^32 - 1)).
 */
#define HHT_FAULT_NONE 0
#define HHT_FAULT_WITHHOLD_SCAN_TILE 1
#define HHT_FAULT_GRAPH_CAPACITY 2
int hht_inject_fault(hht_ctx *ctx, int32_t kind, int64_t arg);

/* Short description of an HHT_* code (static string). */
const char *hht_strerror(int code);

/* Library build description (static string). */
const char *hht_version(void);

#ifdef __cplusplus
}
#endif

#endif /* HHT_H_ */
