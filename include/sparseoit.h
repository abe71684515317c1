/*
 * sparseoit.h -- C ABI of libsparseoit, the GB300 (sm_103a) implementation
 * of SparseOIT's differentiable order-independent-transparency Gaussian
 * splat renderer restricted to an active set of splats (arXiv 2605.13855).
 *
 * What is computed (paper references are to sections / equations /
 * algorithms of the paper):
 *   - Eq. 7 (weighted-blended OIT):  C = T c0 + (1 - T) P / Q,
 *       P = sum_i c_i a_i w_i,  Q = sum_i a_i w_i,  T = prod_i (1 - a_i),
 *     with the per-pixel opacity a_i of Eq. 5, the 2D covariance of Eq. 6
 *     (from Sigma = R S S^T R^T, Eq. 2), the degree-3 SH colour of Eq. 4 and
 *     the OIT weight w = max(0, 1 - d/sigma) v(r) of Eq. 1.
 *   - Sec. 4.1 (active set): only splats in the active set A are projected,
 *     binned and accumulated each iteration; the frozen complement's
 *     per-pixel sums (P, Q, log T) sit in device buffers, one per training
 *     view, and are combined with A's sums (P = P_A + P_F, Q = Q_A + Q_F,
 *     T = T_A exp(logT_F)).  Their update after an active-set change is
 *     delayed until the view is used (Sec. 4.1 "Implementation Details",
 *     Alg. 2 "BAU").
 *   - App. A / Alg. 2: binning by tile id only (no depth sort).
 *   - App. B / Eq. 9-10 and Sec. 4.2: backward pass; only A's parameters
 *     receive gradients.
 *
 * Conventions shared by every call:
 *   - Every function returns 0 (SPARSEOIT_OK) or a negative error code and
 *     never throws or aborts; sparseoit_last_error() then describes it.
 *   - `stream` is a cudaStream_t (passed as void* so this header needs no
 *     CUDA include).  Work is enqueued on it and the call returns without
 *     waiting, except where a call says it synchronises.
 *   - Pointers documented "device" must be device (or managed) memory that
 *     the caller owns and keeps alive until the enqueued work completes.
 *     "host" pointers are read before the call returns.
 *   - Arrays are dense, row-major, 32-bit float unless stated.
 *   - Pixel (x, y) of a W x H view has its centre at (x + 0.5, y + 0.5);
 *     images are [H, W, 3] (HWC).
 *   - The context owns its workspace (projected records, tile bins, pixel
 *     states, frozen sums); it is allocated with cudaMalloc on the current
 *     device in sparseoit_create / sparseoit_set_active and grown there when
 *     needed.  One context must not be used from two host threads at once.
 */
#ifndef SPARSEOIT_H
#define SPARSEOIT_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define SPARSEOIT_ABI_VERSION 1
#define SPARSEOIT_MAX_BATCH_VIEWS 32   /* views in one forward / backward call */

/* Error codes. */
enum {
    SPARSEOIT_OK = 0,
    SPARSEOIT_ERR_INVALID_ARG = -1,  /* a null / out-of-range argument            */
    SPARSEOIT_ERR_OOM = -2,          /* cudaMalloc failed                          */
    SPARSEOIT_ERR_CUDA = -3,         /* a CUDA runtime call or launch failed       */
    SPARSEOIT_ERR_STATE = -4,        /* call out of order: forward on a view whose
                                        frozen sums are stale, backward without a
                                        forward, forward before set_active         */
    SPARSEOIT_ERR_CAPACITY = -5,     /* the (splat, tile) pair arena overflowed;
                                        outputs of that call are invalid; enlarge
                                        it with sparseoit_reserve_pairs and redo   */
    SPARSEOIT_ERR_TIMEOUT = -6       /* a bounded device-side wait gave up         */
};

/* Storage type of the SH coefficient arrays. */
enum { SPARSEOIT_F32 = 0, SPARSEOIT_BF16 = 1 };

/* Frozen-sum update modes (sparseoit_commit_frozen). */
enum {
    SPARSEOIT_COMMIT_INCREMENTAL = 0, /* add D+ = A_old \ A_new, subtract D- = A_new \ A_old */
    SPARSEOIT_COMMIT_RECOMPUTE = 1    /* re-render the whole complement of A                */
};

typedef struct sparseoit_ctx sparseoit_ctx;

/* Pinhole camera.  A world point X maps to the camera-space point
 * t_c = R X + t (x right, y down, z forward) and to the pixel
 * (fx t_c.x / t_c.z + cx, fy t_c.y / t_c.z + cy).  Splats with t_c.z <= 0.2
 * are culled.  width / height must equal the view's size given at create. */
typedef struct {
    float R[9];          /* world -> camera rotation, row-major */
    float t[3];
    float fx, fy, cx, cy;
    int32_t width, height;
} sparseoit_camera;

/* The splat parameters (Sec. 3.1 / 3.2), device pointers, n rows each.
 * rows = SPARSEOIT_ROWS_BY_SPLAT: row i is splat i, n = max_splats (the
 * full set G).  rows = SPARSEOIT_ROWS_ACTIVE: row r is the r-th active splat
 * in the order of sparseoit_get_active, n = |A| -- the layout of an active
 * stage (sparseoit_gather_active), read with coalesced row loads; accepted
 * by sparseoit_forward / backward / autotune only (the frozen-sum commit
 * and the active-set update need every splat). */
#define SPARSEOIT_ROWS_BY_SPLAT 0
#define SPARSEOIT_ROWS_ACTIVE 1
typedef struct {
    const float *means;           /* [n, 3] centre mu                                 */
    const float *quats;           /* [n, 4] rotation quaternion (w, x, y, z), any norm */
    const float *log_scales;      /* [n, 3] log of the axis scales s                  */
    const float *opacity_logits;  /* [n]    opacity o = sigmoid(logit)                */
    const void *sh_color;         /* [n, 16, 3] colour SH h (degree 3), sh_dtype      */
    const void *sh_weight;        /* [n, 16] OIT-weight SH v (single channel)         */
    int32_t sh_dtype;             /* SPARSEOIT_F32 or SPARSEOIT_BF16                  */
    float sigma;                  /* scene depth scale of Eq. 1 (> 0)                 */
    float bg[3];                  /* background colour c0 of Eq. 7                    */
    int64_t n;                    /* number of rows (max_splats, or |A| for ROWS_ACTIVE) */
    int32_t rows;                 /* SPARSEOIT_ROWS_BY_SPLAT or SPARSEOIT_ROWS_ACTIVE */
    int32_t reserved;
} sparseoit_splats;               /* quats, sh_color and sh_weight 16-byte aligned (vector loads) */

/* Gradient outputs, device pointers.  Only active splats receive gradients
 * (Sec. 4.1).  With rows_by_splat == 0 the rows are COMPACT: row r belongs to
 * the r-th active splat in ascending splat index (sparseoit_get_active) and
 * the arrays have n_active rows.  With rows_by_splat != 0 the arrays have n
 * rows, an active splat's gradient goes to the row of its splat index and
 * the rows of inactive splats are not written.  FP32 regardless of sh_dtype;
 * quats, sh_color and sh_weight 16-byte aligned.  The active rows (and
 * *sigma) are overwritten by sparseoit_backward, or added to with
 * accumulate != 0. */
typedef struct {
    float *means;           /* [n_active, 3]     */
    float *quats;           /* [n_active, 4]     */
    float *log_scales;      /* [n_active, 3]     */
    float *opacity_logits;  /* [n_active]        */
    float *sh_color;        /* [n_active, 16, 3] */
    float *sh_weight;       /* [n_active, 16]    */
    float *sigma;           /* [1]: dL/dsigma summed over active splats and views */
    int32_t rows_by_splat;  /* 0: compact rows, else rows indexed by splat index */
    int32_t accumulate;     /* 0: overwrite the active rows and *sigma; else add to them
                               (sum the gradients of several backward calls)        */
} sparseoit_grads;

/* Launch configuration (NULL = defaults). */
typedef struct {
    int64_t max_pairs;      /* capacity of the (splat, tile) pair arena shared by
                               the views of one call; 0 = 1 << 25               */
    int32_t fwd_pixels_per_thread; /* forward raster: pixels per thread, 1, 2 or 4
                                      (256 / 128 / 64 threads per 16x16 tile);
                                      0 = default (4)                          */
    int32_t proj_lanes_per_splat;  /* projection: lanes per splat, 1, 2, 4 or
                                      16; 0 = default (4)                      */
    int32_t bwd_walk;              /* per-splat backward raster: the order in
                                      which warps take a tile's splats.
                                      0 = default = 1; 1 = sorted in shared
                                      memory by the first tile row the
                                      splat's ellipse reaches (whole-tile
                                      splats first); 2 = arena order        */
    int32_t raster_tile_order;     /* rasters take tiles heaviest first (tiles
                                      ranked by pair count in four classes per
                                      octave) instead of in index order;
                                      1 = on, -1 = off, 0 = default (on)       */
    int32_t bwd_parallel;          /* backward raster organisation (the
                                      ablation of Sec. 5.3, Tab. 2):
                                      0 = default = 1; 1 = per splat (a lane
                                      per splat, pixel states in shared
                                      memory, one atomic set per splat and
                                      tile); 2 = per pixel, warp-reduced
                                      atomics; 3 = per pixel, one atomic set
                                      per contributing pair (3DGS)          */
    int32_t raster_persistent;     /* rasters (forward, backward, frozen-sum
                                      commit) as persistent blocks, as many
                                      as fit on the device, that take the
                                      tiles of a call from an atomic queue in
                                      the raster order; 1 = on, -1 = off,
                                      0 = default (off)                      */
} sparseoit_config;

/* Create a context for a scene of max_splats splats and n_views training
 * views of sizes view_w[k] x view_h[k] (host arrays, 1 <= n_views).
 * Allocates the per-view frozen sums (5 floats per pixel: P_r, P_g, P_b, Q,
 * log T) and the pixel states.  *out receives the context. */
int sparseoit_create(sparseoit_ctx **out, int64_t max_splats, int32_t n_views, const int32_t *view_w,
                     const int32_t *view_h, const sparseoit_config *cfg);

/* Release every buffer of the context (synchronises the device). */
int sparseoit_destroy(sparseoit_ctx *ctx);

/* Sec. 4.1: set the active set A from a device mask d_mask[n] (nonzero =
 * active; n == max_splats).  Compacts the mask into the ascending active
 * index list and records the deltas D+ = A_old \ A_new and D- = A_new \ A_old
 * against the previous mask for the delayed frozen-sum update.  Every view
 * becomes stale until sparseoit_commit_frozen.  SYNCHRONISES `stream` (the
 * host needs |A| to size later launches). */
int sparseoit_set_active(sparseoit_ctx *ctx, const uint8_t *d_mask, int64_t n, void *stream);

/* Sec. 4.1, the same update of A without waiting: the compaction and the
 * copy of the four set sizes to host memory are enqueued on `stream` and the
 * call returns.  The first later call on this context that needs the sizes
 * (every call that takes splats, sparseoit_get_active, sparseoit_adam_step,
 * sparseoit_gather_active / sparseoit_scatter_active, the next
 * set_active) waits for that copy alone, so the host can prepare the next
 * step meanwhile.  d_mask must stay valid and unchanged until `stream` has
 * run the compaction.  Same arguments and errors as sparseoit_set_active;
 * an error of the compaction itself surfaces at that later wait. */
int sparseoit_set_active_async(sparseoit_ctx *ctx, const uint8_t *d_mask, int64_t n, void *stream);

/* The active index list (device, ascending, int32) and |A|.  The pointer
 * stays valid until the next set_active. */
int sparseoit_get_active(sparseoit_ctx *ctx, const int32_t **d_idx, int64_t *n_active);

/* Sec. 4.1 / Alg. 2 (BAU): bring the frozen sums of `view` up to date with
 * the current active set, for camera *cam (host struct).  INCREMENTAL is
 * exact when the view was last committed under the previous active set and
 * the splats of the complement (and sigma, c0, the camera) did not change
 * since; otherwise the call falls back to RECOMPUTE.  A view that is
 * already current is left as it is. */
int sparseoit_commit_frozen(sparseoit_ctx *ctx, const sparseoit_splats *splats, const sparseoit_camera *cam,
                            int32_t view, int32_t mode, void *stream);

/* Device pointer to the frozen sums of `view`: 5 planes of H*W floats
 * (P_r, P_g, P_b, Q, log T).  Valid until destroy. */
int sparseoit_get_frozen(sparseoit_ctx *ctx, int32_t view, float **d_planes);

/* Sec. 4.1 keeps the pre-rendered sums of the inactive splats as the only
 * state that outlives an iteration; this restores them (checkpoint and
 * resume).  planes: 5 planes of H*W floats in the layout of
 * sparseoit_get_frozen, in device or host memory (copied with
 * cudaMemcpyDefault on `stream`; the caller keeps ownership, and the planes
 * must stay valid and unchanged until `stream` has completed the copy --
 * with pinned host memory the copy is truly asynchronous).  The view is
 * then treated as committed under the current active set: the caller
 * guarantees that the planes are the sums of the complement of that set
 * (for example saved by sparseoit_get_frozen under the same mask) for the
 * current parameters of the complement, sigma, c0 and the view's camera.
 * ERR_STATE before the first set_active; ERR_INVALID_ARG for a bad view or
 * a null pointer; ERR_CUDA if the copy cannot be enqueued. */
int sparseoit_set_frozen(sparseoit_ctx *ctx, int32_t view, const float *planes, void *stream);

/* Alg. 1 / Alg. 2 (BAN): render the active set of n_views views in one
 * batched launch sequence and compose each with its frozen sums (Eq. 7).
 *   cams[k] (host) is the camera of view views[k] (host int array);
 *   d_images[k] (device [H, W, 3]) receives the image of view views[k].
 *   d_targets: NULL, or n_views device images [H, W, 3].  With targets the
 *     L1 loss  L = sum_k mean_{pixels, channels} |C_k - I_k|  is written to
 *     d_loss (device float, overwritten) and the backward needs no
 *     d_grad_images (dL/dC = sign(C - I) / (3 H W), sign(0) = 0).
 * Every listed view must be committed under the current active set, else
 * SPARSEOIT_ERR_STATE.  1 <= n_views <= SPARSEOIT_MAX_BATCH_VIEWS, no view
 * listed twice. */
int sparseoit_forward(sparseoit_ctx *ctx, const sparseoit_splats *splats, const sparseoit_camera *cams,
                      const int32_t *views, int32_t n_views, float *const *d_images, const float *const *d_targets,
                      float *d_loss, void *stream);

/* App. B / Sec. 4.2: gradients of the last forward's loss with respect to the
 * active splats' parameters (summed over its views).  d_grad_images: NULL
 * when that forward had targets (fused L1), else n_views device arrays
 * [H, W, 3] holding dL/dC in the forward's view order.  `splats` must be the
 * same parameter values as in the forward.  After a forward with targets (or
 * sparseoit_loss_l1_dssim) the call may be repeated; after a forward without
 * targets it turns that forward's planes into the backward state in place, so a
 * second backward (or a loss) of the same forward returns SPARSEOIT_ERR_STATE. */
int sparseoit_backward(sparseoit_ctx *ctx, const sparseoit_splats *splats, const float *const *d_grad_images,
                       sparseoit_grads *out, void *stream);

/* Result of sparseoit_autotune. */
typedef struct {
    int32_t fwd_pixels_per_thread;   /* chosen forward strip (1, 2 or 4)              */
    int32_t n_candidates;
    int32_t candidates[4];           /* the strips tried                              */
    float ms[4];                     /* mean forward time of each strip (one block
                                        per tile)                                     */
    int32_t fwd_persistent;          /* chosen: 1 = persistent forward raster blocks  */
    float fwd_persistent_ms;         /* mean forward time, chosen strip, persistent   */
    int32_t bwd_walk;                /* chosen backward splat order (1 sorted by first
                                        row, 2 arena order); 0 = not tuned (the
                                        forward had no targets)                       */
    int32_t bwd_persistent;          /* chosen: 1 = persistent backward raster blocks */
    float bwd_ms[4];                 /* mean backward-raster time: sorted, arena,
                                        sorted persistent, arena persistent            */
} sparseoit_tuning;

/* Autotuner over the launch options that matter on a given batch (the tile
 * stays 16x16: the binning, both rasters and the pixel state are built on
 * it).  It times, on this exact batch -- the arguments are those of
 * sparseoit_forward, which it runs -- (1) the forward raster's per-thread
 * pixel strip (1x1, 1x2 and 1x4 pixels, i.e. 256 / 128 / 64 threads per
 * tile), then the chosen strip as persistent blocks taking tiles from a
 * queue; and, when targets are given (fused L1, so the pixel state exists),
 * (2) the backward raster with the tile's splats sorted by first row or in
 * arena order, each as one block per tile and as persistent blocks.  Each
 * candidate: 1 warm-up + `reps` timed runs, CUDA events on `stream`.  The
 * fastest of each is kept for later calls, a persistent raster only if it is
 * at least 2 % faster than one block per tile.  The outputs of the last call are
 * valid forward outputs (a backward must follow it as after any forward).
 * Synchronises `stream`; not for use during stream capture. */
int sparseoit_autotune(sparseoit_ctx *ctx, const sparseoit_splats *splats, const sparseoit_camera *cams,
                       const int32_t *views, int32_t n_views, float *const *d_images, const float *const *d_targets,
                       float *d_loss, int32_t reps, sparseoit_tuning *out, void *stream);

/* Enlarge the pair arena to at least max_pairs entries (synchronises). */
int sparseoit_reserve_pairs(sparseoit_ctx *ctx, int64_t max_pairs);

/* Synchronise `stream`, read and clear the device status word.  Returns
 * SPARSEOIT_ERR_CAPACITY if a pair arena overflowed since the last call,
 * SPARSEOIT_ERR_TIMEOUT if a bounded wait gave up, else SPARSEOIT_OK. */
int sparseoit_status(sparseoit_ctx *ctx, void *stream);

/* Failure injection for tests of the bounded device-side wait (Alg. 2's
 * binning scan, IdentifyTileRanges, run as a single-pass scan with look-back
 * over partitions of 1024 tiles): in the next binning of this context
 * (a forward, a commit or an update), partition `partition` of the tile
 * scan posts nothing, so every later partition runs out its wait (0.25 s)
 * and sets the timeout flag; the kernels after the scan then do nothing and
 * sparseoit_status returns SPARSEOIT_ERR_TIMEOUT.  The outputs of that call
 * are invalid; the context stays usable and the next call runs normally.
 * A partition number at or past the last partition has no effect.  The
 * injection is consumed by the next binning. */
int sparseoit_inject_scan_stall(sparseoit_ctx *ctx, int32_t partition);

/* Counters of the last forward (synchronises `stream`): number of
 * (splat, tile) pairs binned (M, summed over its views) and the number of
 * (splat, pixel) pairs with alpha >= 1/255 (E, counted by the forward
 * raster when counting is enabled with sparseoit_set_counting). */
int sparseoit_last_counts(sparseoit_ctx *ctx, void *stream, int64_t *n_pairs, int64_t *n_contrib);

/* Enable (1) / disable (0) the contributing-pair counter of the forward
 * raster (off by default; costs one atomic per thread block). */
int sparseoit_set_counting(sparseoit_ctx *ctx, int32_t enable);

/* Per-kernel device time, accumulated while profiling is enabled. */
typedef struct {
    char name[32];          /* kernel name                                   */
    int64_t launches;       /* launches timed since the last get_profile     */
    double total_ms;        /* summed CUDA-event durations of those launches */
} sparseoit_kernel_time;

/* Enable (1) / disable (0) profiling: every kernel launch of the library is
 * bracketed by CUDA events recorded on the launching stream.  Must be off
 * while a stream is being captured into a CUDA graph. */
int sparseoit_set_profiling(sparseoit_ctx *ctx, int32_t enable);

/* Synchronise on the recorded events and return the per-kernel totals since
 * the previous call (then reset).  Writes at most max_entries entries to out
 * (host array) and their number to *n_out. */
int sparseoit_get_profile(sparseoit_ctx *ctx, int32_t max_entries, sparseoit_kernel_time *out, int32_t *n_out);

/* Last error message of the context (or of the last failed create when ctx
 * is NULL).  Never NULL. */
const char *sparseoit_last_error(const sparseoit_ctx *ctx);

/* SPARSEOIT_ABI_VERSION of the loaded library. */
int sparseoit_version(void);

/* Sec. 4.1, "Updating Active Set via Subsampling" (Alg. 1, the
 * IsActiveUpdateIteration branch): farthest point sampling of s of the n
 * training views by camera centre c = -R^T t.  cams: host [n]; first: the
 * randomly drawn starting view (the caller draws it and passes it in);
 * out: host int32 [s].  out[0] = first; each next entry is the view whose
 * (double precision) distance to the nearest view chosen so far is largest
 * (ties: lowest index).  Host only, no device work; 1 <= s <= n and
 * 0 <= first < n, else SPARSEOIT_ERR_INVALID_ARG. */
int sparseoit_fps_views(const sparseoit_camera *cams, int32_t n, int32_t s, int32_t first, int32_t *out);

/* Eq. 8, read as "active if at least one attribute is active" (the text
 * after Eq. 8): per splat i < n, the Euclidean norms of the gradient of
 * each attribute group -- mu (3), q (4), log s (3), opacity logit (1),
 * colour SH h (48), weight SH w (16) -- and d_mask[i] = 1 if some group's
 * norm exceeds its threshold eps[k] (host float[6], that order), else 0.
 * g: gradients in full rows indexed by splat (the rows_by_splat layout of
 * sparseoit_backward; device pointers, FP32; g->sigma is not read);
 * d_mask: device u8[n]; d_norms: device float [n,6] receiving the norms,
 * or NULL.  The norms are summed in FP32 in a fixed order.  Asynchronous
 * on `stream`. */
int sparseoit_activeness(const sparseoit_grads *g, int64_t n, const float *eps, uint8_t *d_mask, float *d_norms,
                         void *stream);

/* The whole periodic active-set update of Alg. 1 on the context: picks
 * n_sub of the n_views training views by sparseoit_fps_views (from
 * `first`); for each picked view j renders the whole splat set (every
 * splat, no frozen sums) with the fused L1 loss against d_targets[j]
 * (device FP32 [H_j, W_j, 3]) and back-propagates, summing the gradients of
 * the n_sub view losses into `scratch` (full rows indexed by splat, device
 * FP32, overwritten; scratch->sigma receives the summed dL/dsigma).  The
 * current active set and the views' frozen sums are not touched by these
 * renders.  Then sparseoit_activeness(scratch, eps) writes the new mask to
 * d_mask (device u8[max_splats]) and the call ends with
 * sparseoit_set_active(d_mask): every view is stale afterwards, and a view
 * committed under the previous active set is brought up to date by an
 * INCREMENTAL commit of the changes (the delayed update of Sec. 4.1).
 * cams: host [n_views], the context's views in order (view k has the
 * context's size k); sel_out: host int32 [n_sub] (nullable) receives the
 * picked views.  Synchronises `stream` (set_active does). */
int sparseoit_update_active_set(sparseoit_ctx *ctx, const sparseoit_splats *splats, const sparseoit_camera *cams,
                                int32_t n_views, const float *const *d_targets, int32_t n_sub, int32_t first,
                                const float *eps, sparseoit_grads *scratch, uint8_t *d_mask, int32_t *sel_out,
                                void *stream);

/* The photometric loss of 3DGS, which the paper keeps (Sec. 5.1):
 * L = sum over the views of the last forward of
 *     (1 - lambda) mean|C - I| + lambda (1 - SSIM(C, I)),
 * SSIM per colour channel with an 11 x 11 Gaussian window (sigma 1.5), zero
 * padding, C1 = 0.01^2, C2 = 0.03^2, averaged over pixels and channels (3DGS
 * uses lambda = 0.2).  Call it after a sparseoit_forward without targets: it
 * reads that forward's images, writes *d_loss (device float), optionally the
 * image gradients dL/dC to d_grad_images[k] (host array of device [H, W, 3]
 * FP32 pointers, or NULL), and leaves the pixel state so that
 * sparseoit_backward(..., d_grad_images = NULL, ...) back-propagates L.
 * d_targets: host array of device [H, W, 3] FP32 pointers, one per view of
 * the forward; bg: host float[3], the background of that forward.
 * ERR_STATE if there is no such forward (or its state was already used). */
int sparseoit_loss_l1_dssim(sparseoit_ctx *ctx, const float *const *d_targets, float lambda, float *d_loss,
                            float *const *d_grad_images, const float *bg, void *stream);

/* A set of FP32 per-splat row arrays (parameters or Adam moments), device
 * pointers, rows indexed by splat: means [N,3], quats [N,4], log_scales
 * [N,3], opacity_logits [N], sh_color [N,16,3], sh_weight [N,16], and the
 * scene scalar sigma [1]. */
typedef struct {
    float *means, *quats, *log_scales, *opacity_logits, *sh_color, *sh_weight;
    float *sigma;
} sparseoit_rows;

/* Adam hyper-parameters (Sec. 5.1 "Implementation Details": Adam; learning
 * rates of o, sigma and v from the paper, the rest the caller's). */
typedef struct {
    float lr[8];      /* means, quats, log_scales, opacity_logits, sh_color degree 0, sh_color degrees 1-3,
                         sh_weight, sigma */
    float beta1, beta2, eps;
    int32_t step;     /* t >= 1: the bias corrections are 1 - beta^t */
    int32_t rows;     /* layout of params, m and v: SPARSEOIT_ROWS_BY_SPLAT (N rows) or
                         SPARSEOIT_ROWS_ACTIVE (|A| rows in active order, like the gradients) */
} sparseoit_adam;

/* Sparse Adam over the active set: for every active splat (the context's
 * active index list, in its order) and every parameter element,
 *   m = b1 m + (1 - b1) g,  v = b2 v + (1 - b2) g^2,
 *   p -= (lr / (1 - b1^t)) m / (sqrt(v) / sqrt(1 - b2^t) + eps)
 * (the torch.optim.Adam step).  grads: the compact rows of the last
 * sparseoit_backward (rows_by_splat = 0, N_A rows in active order; grads->sigma
 * = dL/dsigma); params, m, v: rows by splat or active rows (cfg->rows),
 * updated in place; rows of inactive splats are neither read nor written.  sigma (params,
 * m, v ->sigma, all non-null or all null) is updated with lr[7].  The
 * caller copies the new sigma into sparseoit_splats.sigma (a host value)
 * before the next forward, and recommits the frozen sums if it changed.
 * Asynchronous on `stream`. */
int sparseoit_adam_step(sparseoit_ctx *ctx, const sparseoit_grads *grads, sparseoit_rows *params, sparseoit_rows *m,
                        sparseoit_rows *v, const sparseoit_adam *cfg, void *stream);

/* Stage layout (Sec. 4.1: between two active-set updates only A is
 * optimised): copy the active rows of a full row set (rows by splat) into
 * active rows (|A| rows in active order), or back.  FP32 arrays except
 * sh_color / sh_weight, whose element type is sh_dtype; the sigma fields
 * are not read.  Asynchronous on `stream`. */
int sparseoit_gather_active(sparseoit_ctx *ctx, const sparseoit_rows *full, sparseoit_rows *active, int32_t sh_dtype,
                            void *stream);
int sparseoit_scatter_active(sparseoit_ctx *ctx, const sparseoit_rows *active, sparseoit_rows *full, int32_t sh_dtype,
                             void *stream);

/* Allocation-free active-index compaction.  The paper has no counterpart:
 * this entry point serves callers that cannot allocate device memory --
 * code that must not trigger the device-wide synchronisation that
 * cudaMalloc / cudaFree imply, plug-ins running inside another runtime that
 * owns the whole device memory budget, and deployments that forbid
 * allocation after start-up.  It writes to d_idx (device, int32, room for n
 * entries) the ascending indices i with d_mask[i] != 0 (d_mask: device, n
 * bytes) and their number to *d_count (device int64), the same list that
 * sparseoit_set_active / sparseoit_get_active produce, without a context.
 * Its block-count scratch is a fixed file-scope device array of
 * SPARSEOIT_STATIC_MAX_SPLATS / 4096 ints (16 KiB) that every GPU loading the
 * library keeps until the process exits; it calls no cudaMalloc, cudaFree or
 * other allocating routine.  n > SPARSEOIT_STATIC_MAX_SPLATS (or a null
 * pointer) returns SPARSEOIT_ERR_INVALID_ARG without enqueuing work.  All
 * calls share that scratch, so calls that overlap on the GPU (other streams
 * or host threads on the same device) race and must be serialised by the
 * caller; each call writes every scratch slot it reads, so no clearing is
 * needed.  The first call on a device looks up the scratch address with
 * cudaGetSymbolAddress for the current device: make it before any stream
 * capture.  That address is kept for the rest of the process, so do not
 * reset the device (cudaDeviceReset) or destroy its primary context between
 * calls.  Asynchronous on `stream`. */
#define SPARSEOIT_STATIC_MAX_SPLATS (16 * 1024 * 1024)
int sparseoit_compact_active_static(const uint8_t *d_mask, int64_t n, int32_t *d_idx, int64_t *d_count,
                                    void *stream);

#ifdef __cplusplus
}
#endif
#endif /* SPARSEOIT_H */
