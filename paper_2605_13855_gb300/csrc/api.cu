// api.cu -- the C ABI of libsparseoit (declared in include/sparseoit.h).
//
// A context holds the active-set state (masks, compacted index lists and
// the deltas of the last change), one set of frozen sums per training view
// with the active-set generation it was committed under, and the workspace
// of one batched forward / backward: projected records, tile counts /
// offsets, the pair arena, the pixel states and the screen-space gradients.
#include <cstdio>
#include <cstring>
#include <map>
#include <cmath>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "../../include/sparseoit.h"
#include "common.cuh"
#include "launch.h"

namespace {
// A named NVTX range around each entry point that enqueues GPU work, so that a
// profiler timeline shows the library's calls (header-only NVTX; inert when no
// tool is attached).
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange &) = delete;
    NvtxRange &operator=(const NvtxRange &) = delete;
};
}  // namespace

using namespace soit;

struct sparseoit_ctx {
    int64_t N = 0;
    int n_views = 0;
    std::vector<int> W, H;
    int64_t pair_cap = 0;
    int fwd_strip = 4;            // pixels per thread of the forward raster
    int proj_lanes = 4;           // lanes per splat of the projection
    int bwd_walk = kBwdWalkSorted; // backward raster: pairs sorted by first row, or arena order
    bool tile_order = true;       // rasters take tiles heaviest first
    int bwd_parallel = 1;         // 1 per splat, 2 per pixel warp-reduced, 3 per pixel per-pair atomics
    std::string err;

    // active set
    uint8_t *d_mask[2] = {nullptr, nullptr};
    int cur = 0;
    int *d_idx_active = nullptr, *d_idx_comp = nullptr, *d_idx_plus = nullptr, *d_idx_minus = nullptr;
    int *d_blk = nullptr;
    int64_t *d_totals = nullptr;
    int64_t *h_totals = nullptr;  // pinned
    int64_t n_active = 0, n_comp = 0, n_plus = 0, n_minus = 0;
    // set by sparseoit_set_active_async: the counts above are still being copied into h_totals;
    // ev_counts completes with the copy
    bool counts_pending = false;
    cudaEvent_t ev_counts = nullptr;
    int64_t generation = 0;       // number of set_active calls
    bool have_mask = false;
    std::vector<int64_t> view_gen;
    std::vector<float *> d_frozen;

    // batch workspace
    float4 *d_rec = nullptr, *d_ext = nullptr;
    int64_t rec_cap = 0;          // records
    int *d_tile_count = nullptr, *d_offsets = nullptr, *d_cursor = nullptr, *d_order = nullptr;
    int64_t tile_cap = 0;
    uint32_t *d_pairs = nullptr;
    std::vector<float *> d_state;  // per batch slot, 5 planes of the largest view
    int64_t max_pix = 0;
    float4 *d_sgrad = nullptr;
    int64_t sgrad_cap = 0;        // records
    bool sgrad_clean = false;     // zeroed by the last forward's projection, no backward since
    float *d_sig_part = nullptr;  // dL/dsigma partials, one per block of the backward chain
    int64_t sig_part_cap = 0;
    unsigned *d_sig_count = nullptr;  // the chain's finished-block counter (zero between launches)
    unsigned *d_status = nullptr;
    void *d_scan = nullptr;        // binning scan scratch (ScanScratch), zeroed before each scan
    int *d_queue = nullptr;        // tile queues of the persistent rasters (forward, backward)
    bool fwd_persistent = false;   // forward / sums raster as persistent blocks over a tile queue
    bool bwd_persistent = false;   // backward raster as persistent blocks over a tile queue
    int scan_withhold = -1;        // failure injection: the next scan's partition that posts nothing
    int64_t *d_npairs = nullptr;
    unsigned long long *d_contrib = nullptr;
    bool counting = false;
    float *d_ssim_abc = nullptr;   // D-SSIM: 9 partials per pixel of the largest view
    double *d_ssim_sums = nullptr; // D-SSIM: 2 sums per view of a batch
    float *d_upd_image = nullptr;  // image and loss of the active-set update's full-set renders
    float *d_upd_loss = nullptr;

    // profiling: events bracketing every launch while enabled
    bool profiling = false;
    struct Mark { const char *name; cudaEvent_t a, b; };
    std::vector<Mark> marks;
    std::vector<cudaEvent_t> event_pool;

    // last forward
    bool have_fwd = false;
    bool last_fused = false;
    // a backward after a forward without targets turned its (F, T, Q) planes into the backward
    // state in place: another backward or loss needs a new forward
    bool planes_consumed = false;
    Batch last_batch;
    int last_n_list = 0;
    const int *last_list = nullptr;  // index list of the last forward (active list or identity)
    int *d_idx_all = nullptr;        // identity list 0..N-1 (full-set renders of the active-set update)
    int64_t last_generation = -1;
};

static std::string g_create_err;

static int fail(sparseoit_ctx *c, int code, const std::string &msg) {
    if (c) c->err = msg; else g_create_err = msg;
    return code;
}

static int cuda_check(sparseoit_ctx *c, cudaError_t e, const char *what) {
    if (e == cudaSuccess) return SPARSEOIT_OK;
    const int code = (e == cudaErrorMemoryAllocation) ? SPARSEOIT_ERR_OOM : SPARSEOIT_ERR_CUDA;
    return fail(c, code, std::string(what) + ": " + cudaGetErrorString(e));
}

static cudaEvent_t take_event(sparseoit_ctx *ctx) {
    if (!ctx->event_pool.empty()) {
        cudaEvent_t e = ctx->event_pool.back();
        ctx->event_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
    return e;
}

// Brackets one kernel launch with events on its stream when profiling.
struct ProfScope {
    sparseoit_ctx *ctx;
    const char *name;
    cudaStream_t st;
    cudaEvent_t a = nullptr;
    ProfScope(sparseoit_ctx *c, const char *n, cudaStream_t s) : ctx(c), name(n), st(s) {
        if (ctx->profiling) {
            a = take_event(ctx);
            if (a) cudaEventRecord(a, st);
        }
    }
    ~ProfScope() {
        if (!a) return;
        cudaEvent_t b = take_event(ctx);
        if (!b) { ctx->event_pool.push_back(a); return; }
        cudaEventRecord(b, st);
        ctx->marks.push_back({name, a, b});
    }
};

#define CK(call, what)                                              \
    do {                                                            \
        int rc__ = cuda_check(ctx, (call), what);                   \
        if (rc__ != SPARSEOIT_OK) return rc__;                      \
    } while (0)

#define CK_LAUNCH(what) CK(cudaGetLastError(), what)

template <typename T>
static cudaError_t grow(T **p, int64_t *cap, int64_t want) {
    if (*p && *cap >= want) return cudaSuccess;
    if (*p) cudaFree(*p);
    *p = nullptr;
    *cap = 0;
    const int64_t n = want > 0 ? want : 1;
    cudaError_t e = cudaMalloc((void **)p, (size_t)n * sizeof(T));
    if (e == cudaSuccess) *cap = n;
    return e;
}

// The host copies of |A|, |complement|, |D+|, |D-|: after sparseoit_set_active_async they are
// still in flight, and the first call that needs them waits here for the copy.
static int sync_counts(sparseoit_ctx *ctx) {
    if (!ctx->counts_pending) return SPARSEOIT_OK;
    ctx->counts_pending = false;
    CK(cudaEventSynchronize(ctx->ev_counts), "wait for the active-set counts");
    ctx->n_active = ctx->h_totals[0];
    ctx->n_comp = ctx->h_totals[1];
    ctx->n_plus = ctx->h_totals[2];
    ctx->n_minus = ctx->h_totals[3];
    return SPARSEOIT_OK;
}

static int check_splats(sparseoit_ctx *ctx, const sparseoit_splats *s, bool allow_active_rows) {
    if (!s) return fail(ctx, SPARSEOIT_ERR_INVALID_ARG, "splats is null");
    {
        const int rc = sync_counts(ctx);
        if (rc) return rc;
    }
    if (s->rows == SPARSEOIT_ROWS_ACTIVE) {
        if (!allow_active_rows)
            return fail(ctx, SPARSEOIT_ERR_INVALID_ARG, "this call needs the splats in rows by splat");
        if (!ctx->have_mask) return fail(ctx, SPARSEOIT_ERR_STATE, "active rows before set_active");
        if (s->n != ctx->n_active) return fail(ctx, SPARSEOIT_ERR_INVALID_ARG, "splats->n differs from |A|");
    } else if (s->rows != SPARSEOIT_ROWS_BY_SPLAT) {
        return fail(ctx, SPARSEOIT_ERR_INVALID_ARG, "unknown splats->rows");
    } else if (s->n != ctx->N) {
        return fail(ctx, SPARSEOIT_ERR_INVALID_ARG, "splats->n differs from max_splats");
    }
    if (!s->means || !s->quats || !s->log_scales || !s->opacity_logits || !s->sh_color || !s->sh_weight)
        return fail(ctx, SPARSEOIT_ERR_INVALID_ARG, "a splat parameter pointer is null");
    if (((uintptr_t)s->quats & 15u) != 0 || ((uintptr_t)s->sh_color & 15u) != 0 || ((uintptr_t)s->sh_weight & 15u) != 0)
        return fail(ctx, SPARSEOIT_ERR_INVALID_ARG, "quats, sh_color and sh_weight must be 16-byte aligned");
    if (s->sh_dtype != SPARSEOIT_F32 && s->sh_dtype != SPARSEOIT_BF16)
        return fail(ctx, SPARSEOIT_ERR_INVALID_ARG, "unknown sh_dtype");
    if (!(s->sigma > 0.f)) return fail(ctx, SPARSEOIT_ERR_INVALID_ARG, "sigma must be > 0");
    return SPARSEOIT_OK;
}

static SplatPtrs splat_ptrs(const sparseoit_splats *s) {
    SplatPtrs p;
    p.means = s->means;
    p.quats = s->quats;
    p.log_scales = s->log_scales;
    p.opacity_logits = s->opacity_logits;
    p.sh_color = s->sh_color;
    p.sh_weight = s->sh_weight;
    p.sigma = s->sigma;
    for (int k = 0; k < 3; ++k) p.bg[k] = s->bg[k];
    p.active_rows = s->rows == SPARSEOIT_ROWS_ACTIVE ? 1 : 0;
    return p;
}

static int fill_view(sparseoit_ctx *ctx, const sparseoit_camera *cam, int view, ViewDesc &vd, int tile_base) {
    if (!cam) return fail(ctx, SPARSEOIT_ERR_INVALID_ARG, "camera is null");
    if (view < 0 || view >= ctx->n_views) return fail(ctx, SPARSEOIT_ERR_INVALID_ARG, "view index out of range");
    if (cam->width != ctx->W[view] || cam->height != ctx->H[view])
        return fail(ctx, SPARSEOIT_ERR_INVALID_ARG, "camera size differs from the view's size");
    if (!(cam->fx > 0.f) || !(cam->fy > 0.f)) return fail(ctx, SPARSEOIT_ERR_INVALID_ARG, "focal length must be > 0");
    memset(&vd, 0, sizeof(vd));
    memcpy(vd.R, cam->R, sizeof(vd.R));
    memcpy(vd.t, cam->t, sizeof(vd.t));
    vd.fx = cam->fx; vd.fy = cam->fy; vd.cx = cam->cx; vd.cy = cam->cy;
    for (int i = 0; i < 3; ++i)
        vd.campos[i] = -(cam->R[0 * 3 + i] * cam->t[0] + cam->R[1 * 3 + i] * cam->t[1] + cam->R[2 * 3 + i] * cam->t[2]);
    vd.W = cam->width;
    vd.H = cam->height;
    vd.tiles_x = (vd.W + kTile - 1) / kTile;
    vd.tiles_y = (vd.H + kTile - 1) / kTile;
    vd.tile_base = tile_base;
    vd.frozen = ctx->d_frozen[view];
    return SPARSEOIT_OK;
}

// Project list (list1: sign +1, list2: sign -1) into the batch's records and
// bin them by tile.  b.n_list / tile bases must be set.
// Programmatic dependent launch for a kernel that directly follows another of the same call: on
// unless the profiling mode puts event records between the kernels.  Used for the scan, the scatter,
// the backward raster and the backward chain.  Not for the forward rasters: blocks launched early
// take SM slots as the scatter's blocks leave, so the first blocks -- the heaviest tiles -- gather
// on the SMs that free up first (1M splats / 5 %: step 0.385 ms against 0.340 without it).
static bool pdl_ok(const sparseoit_ctx *ctx) { return !ctx->profiling; }

// sgrad_zero (nullable): the screen-space gradient rows, zeroed by the projection for the backward.
static int render_pass_bin(sparseoit_ctx *ctx, Batch &b, const sparseoit_splats *s, const int *list1, int n1,
                           const int *list2, int n2, cudaStream_t st, float4 *sgrad_zero = nullptr) {
    const int64_t nrec = (int64_t)b.n_views * (n1 + n2);
    if (nrec > 0xffffffffll) return fail(ctx, SPARSEOIT_ERR_INVALID_ARG, "too many records in one batch");
    b.tile_order = ctx->tile_order ? ctx->d_order : nullptr;
    b.status = ctx->d_status;
    if (ctx->rec_cap < 3 * nrec || ctx->tile_cap < (int64_t)b.total_tiles + 1)
        return fail(ctx, SPARSEOIT_ERR_STATE, "batch workspace not sized");
    // the scan scratch and the batch's tile counters after it, zeroed together
    CK(cudaMemsetAsync(ctx->d_scan, 0,
                       (size_t)((char *)ctx->d_tile_count - (char *)ctx->d_scan) +
                           (size_t)b.total_tiles * kTileCounterStride * sizeof(int),
                       st),
       "memset(scan scratch, tile counts)");
    const SplatPtrs sp = splat_ptrs(s);
    {
        ProfScope ps(ctx, "project", st);
        launch_project(b, sp, s->sh_dtype == SPARSEOIT_BF16, ctx->proj_lanes, list1, n1, list2, n2, ctx->d_rec,
                       ctx->d_ext, ctx->d_tile_count, sgrad_zero, st);
    }
    CK_LAUNCH("project_kernel");
    {
        ProfScope ps(ctx, "scan_tiles", st);
        launch_scan_tiles(ctx->d_tile_count, b.total_tiles, ctx->d_offsets, ctx->d_cursor,
                          scan_scratch_at(ctx->d_scan, b.total_tiles), ctx->pair_cap, ctx->d_status, ctx->d_npairs,
                          ctx->scan_withhold, pdl_ok(ctx), st);
        ctx->scan_withhold = -1;
    }
    CK_LAUNCH("scan_tiles_kernel");
    {
        ProfScope ps(ctx, "scatter", st);
        launch_scatter(b, ctx->d_rec, ctx->d_ext, ctx->d_cursor, ctx->d_pairs, ctx->pair_cap, ctx->d_tile_count,
                       scan_scratch_at(ctx->d_scan, b.total_tiles), b.tile_order ? ctx->d_order : nullptr, pdl_ok(ctx),
                       st);
    }
    CK_LAUNCH("scatter_kernel");
    return SPARSEOIT_OK;
}

// Records, ext, tile arrays sized for a batch.
static int ensure_batch_ws(sparseoit_ctx *ctx, int64_t nrec, int64_t tiles) {
    if (ctx->rec_cap < 3 * nrec) {
        if (ctx->d_rec) cudaFree(ctx->d_rec);
        if (ctx->d_ext) cudaFree(ctx->d_ext);
        ctx->d_rec = nullptr;
        ctx->d_ext = nullptr;
        ctx->rec_cap = 0;
        const int64_t n = nrec > 0 ? nrec : 1;
        CK(cudaMalloc((void **)&ctx->d_rec, (size_t)(3 * n) * sizeof(float4)), "cudaMalloc(records)");
        CK(cudaMalloc((void **)&ctx->d_ext, (size_t)n * sizeof(float4)), "cudaMalloc(ext)");
        ctx->rec_cap = 3 * n;
    }
    if (ctx->tile_cap < tiles + 1) {
        if (ctx->d_scan) cudaFree(ctx->d_scan);
        if (ctx->d_offsets) cudaFree(ctx->d_offsets);
        if (ctx->d_cursor) cudaFree(ctx->d_cursor);
        if (ctx->d_order) cudaFree(ctx->d_order);
        ctx->d_tile_count = ctx->d_offsets = ctx->d_cursor = ctx->d_order = nullptr;
        ctx->d_scan = nullptr;
        ctx->tile_cap = 0;
        const int64_t n = tiles + 1;
        // the scan scratch with the tile counters after it (256-byte aligned): one memset zeroes both
        const size_t scratch_bytes = (scan_scratch_bytes(n) + 255) & ~(size_t)255;
        CK(cudaMalloc(&ctx->d_scan, scratch_bytes + (size_t)n * kTileCounterStride * sizeof(int)),
           "cudaMalloc(tile counts)");
        ctx->d_tile_count = reinterpret_cast<int *>((char *)ctx->d_scan + scratch_bytes);
        CK(cudaMalloc((void **)&ctx->d_offsets, (size_t)n * sizeof(int)), "cudaMalloc(tile offsets)");
        CK(cudaMalloc((void **)&ctx->d_cursor, (size_t)n * sizeof(int)), "cudaMalloc(tile cursors)");
        CK(cudaMalloc((void **)&ctx->d_order, (size_t)n * sizeof(int)), "cudaMalloc(tile order)");
        // defined contents from the start (a scan that gave up leaves them as they were)
        CK(cudaMemset(ctx->d_offsets, 0, (size_t)n * sizeof(int)), "memset(tile offsets)");
        CK(cudaMemset(ctx->d_cursor, 0, (size_t)n * sizeof(int)), "memset(tile cursors)");
        CK(cudaMemset(ctx->d_order, 0, (size_t)n * sizeof(int)), "memset(tile order)");
        ctx->tile_cap = n;
    }
    return SPARSEOIT_OK;
}

// Mean CUDA-event time of `reps` runs of fn (after one warm-up run) on st.
template <typename F>
static int time_runs(sparseoit_ctx *ctx, cudaStream_t st, int reps, F fn, float *ms_out) {
    cudaEvent_t a = nullptr, b = nullptr;
    CK(cudaEventCreate(&a), "autotune event");
    CK(cudaEventCreate(&b), "autotune event");
    int rc = fn();
    if (!rc) {
        cudaEventRecord(a, st);
        for (int r = 0; r < reps && !rc; ++r) rc = fn();
        cudaEventRecord(b, st);
    }
    float ms = 0.f;
    if (!rc) {
        cudaError_t e = cudaEventSynchronize(b);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, a, b);
        if (e != cudaSuccess) rc = cuda_check(ctx, e, "autotune timing");
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    *ms_out = ms / (float)reps;
    return rc;
}

extern "C" {

int sparseoit_version(void) { return SPARSEOIT_ABI_VERSION; }

const char *sparseoit_last_error(const sparseoit_ctx *ctx) {
    if (!ctx) return g_create_err.c_str();
    return ctx->err.c_str();
}

int sparseoit_create(sparseoit_ctx **out, int64_t max_splats, int32_t n_views, const int32_t *view_w,
                     const int32_t *view_h, const sparseoit_config *cfg) {
    if (!out) return fail(nullptr, SPARSEOIT_ERR_INVALID_ARG, "out is null");
    *out = nullptr;
    if (max_splats < 0 || max_splats > 0x7fffffffll)
        return fail(nullptr, SPARSEOIT_ERR_INVALID_ARG, "max_splats out of range");
    if (n_views < 1 || !view_w || !view_h) return fail(nullptr, SPARSEOIT_ERR_INVALID_ARG, "need >= 1 view");
    for (int v = 0; v < n_views; ++v)
        if (view_w[v] < 1 || view_h[v] < 1 || view_w[v] > 16384 || view_h[v] > 16384)
            return fail(nullptr, SPARSEOIT_ERR_INVALID_ARG, "view size out of range");
    sparseoit_ctx *ctx = new sparseoit_ctx();
    ctx->N = max_splats;
    ctx->n_views = n_views;
    ctx->pair_cap = (cfg && cfg->max_pairs > 0) ? cfg->max_pairs : (int64_t)1 << 25;
    if (cfg && cfg->fwd_pixels_per_thread != 0) {
        const int s = cfg->fwd_pixels_per_thread;
        if (s != 1 && s != 2 && s != 4) {
            delete ctx;
            return fail(nullptr, SPARSEOIT_ERR_INVALID_ARG, "fwd_pixels_per_thread must be 1, 2 or 4");
        }
        ctx->fwd_strip = s;
    }
    if (cfg && cfg->proj_lanes_per_splat != 0) {
        const int l = cfg->proj_lanes_per_splat;
        if (l != 1 && l != 2 && l != 4 && l != 16) {
            delete ctx;
            return fail(nullptr, SPARSEOIT_ERR_INVALID_ARG, "proj_lanes_per_splat must be 1, 2, 4 or 16");
        }
        ctx->proj_lanes = l;
    }
    if (cfg && cfg->bwd_walk != 0) {
        if (cfg->bwd_walk != kBwdWalkSorted && cfg->bwd_walk != kBwdWalkArena) {
            delete ctx;
            return fail(nullptr, SPARSEOIT_ERR_INVALID_ARG, "bwd_walk must be 0, 1 or 2");
        }
        ctx->bwd_walk = cfg->bwd_walk;
    }
    if (cfg && cfg->raster_tile_order != 0) ctx->tile_order = cfg->raster_tile_order > 0;
    if (cfg && cfg->raster_persistent != 0) ctx->fwd_persistent = ctx->bwd_persistent = cfg->raster_persistent > 0;
    if (cfg && cfg->bwd_parallel != 0) {
        if (cfg->bwd_parallel < 1 || cfg->bwd_parallel > 3) {
            delete ctx;
            return fail(nullptr, SPARSEOIT_ERR_INVALID_ARG, "bwd_parallel must be 1, 2 or 3");
        }
        ctx->bwd_parallel = cfg->bwd_parallel;
    }
    if (ctx->pair_cap > 0x7fffffffll) ctx->pair_cap = 0x7fffffffll;
    ctx->view_gen.assign(n_views, -1);
    ctx->d_frozen.assign(n_views, nullptr);
    auto bail = [&](int rc) {
        g_create_err = ctx->err;
        sparseoit_destroy(ctx);
        return rc;
    };
    for (int v = 0; v < n_views; ++v) {
        ctx->W.push_back(view_w[v]);
        ctx->H.push_back(view_h[v]);
        const int64_t hw = (int64_t)view_w[v] * view_h[v];
        if (hw > ctx->max_pix) ctx->max_pix = hw;
        cudaError_t e = cudaMalloc((void **)&ctx->d_frozen[v], (size_t)(5 * hw) * sizeof(float));
        if (e != cudaSuccess) return bail(cuda_check(ctx, e, "cudaMalloc(frozen sums)"));
        e = cudaMemset(ctx->d_frozen[v], 0, (size_t)(5 * hw) * sizeof(float));
        if (e != cudaSuccess) return bail(cuda_check(ctx, e, "cudaMemset(frozen sums)"));
    }
    const int64_t n = max_splats > 0 ? max_splats : 1;
    cudaError_t e = cudaSuccess;
    if (e == cudaSuccess) e = cudaMalloc((void **)&ctx->d_mask[0], (size_t)n);
    if (e == cudaSuccess) e = cudaMalloc((void **)&ctx->d_mask[1], (size_t)n);
    if (e == cudaSuccess) e = cudaMemset(ctx->d_mask[0], 0, (size_t)n);
    if (e == cudaSuccess) e = cudaMemset(ctx->d_mask[1], 0, (size_t)n);
    if (e == cudaSuccess) e = cudaMalloc((void **)&ctx->d_idx_active, (size_t)n * sizeof(int));
    if (e == cudaSuccess) e = cudaMalloc((void **)&ctx->d_idx_comp, (size_t)n * sizeof(int));
    if (e == cudaSuccess) e = cudaMalloc((void **)&ctx->d_idx_plus, (size_t)n * sizeof(int));
    if (e == cudaSuccess) e = cudaMalloc((void **)&ctx->d_idx_minus, (size_t)n * sizeof(int));
    if (e == cudaSuccess) e = cudaMalloc((void **)&ctx->d_blk, (size_t)compact_scratch_ints(n) * sizeof(int));
    if (e == cudaSuccess) e = cudaMalloc((void **)&ctx->d_totals, 4 * sizeof(int64_t));
    if (e == cudaSuccess) e = cudaMallocHost((void **)&ctx->h_totals, 4 * sizeof(int64_t));
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ctx->ev_counts, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaMalloc((void **)&ctx->d_sig_count, sizeof(unsigned));
    if (e == cudaSuccess) e = cudaMemset(ctx->d_sig_count, 0, sizeof(unsigned));
    if (e == cudaSuccess) e = cudaMalloc((void **)&ctx->d_pairs, (size_t)ctx->pair_cap * sizeof(uint32_t));
    if (e == cudaSuccess) e = cudaMalloc((void **)&ctx->d_queue, 2 * sizeof(int));
    if (e == cudaSuccess) e = cudaMalloc((void **)&ctx->d_status, sizeof(unsigned));
    if (e == cudaSuccess) e = cudaMemset(ctx->d_status, 0, sizeof(unsigned));
    if (e == cudaSuccess) e = cudaMalloc((void **)&ctx->d_npairs, sizeof(int64_t));
    if (e == cudaSuccess) e = cudaMemset(ctx->d_npairs, 0, sizeof(int64_t));
    if (e == cudaSuccess) e = cudaMalloc((void **)&ctx->d_contrib, sizeof(unsigned long long));
    if (e == cudaSuccess) e = cudaMemset(ctx->d_contrib, 0, sizeof(unsigned long long));
    if (e != cudaSuccess) return bail(cuda_check(ctx, e, "cudaMalloc(context)"));
    *out = ctx;
    return SPARSEOIT_OK;
}

int sparseoit_destroy(sparseoit_ctx *ctx) {
    if (!ctx) return SPARSEOIT_OK;
    cudaDeviceSynchronize();
    for (float *p : ctx->d_frozen) if (p) cudaFree(p);
    for (float *p : ctx->d_state) if (p) cudaFree(p);
    void *bufs[] = {ctx->d_mask[0], ctx->d_mask[1], ctx->d_idx_active, ctx->d_idx_comp, ctx->d_idx_plus,
                    ctx->d_idx_minus, ctx->d_blk, ctx->d_totals, ctx->d_rec, ctx->d_ext, ctx->d_scan,
                    ctx->d_offsets, ctx->d_cursor, ctx->d_order, ctx->d_queue, ctx->d_pairs, ctx->d_sgrad, ctx->d_status,
                    ctx->d_npairs,
                    ctx->d_contrib, ctx->d_upd_image, ctx->d_upd_loss, ctx->d_ssim_abc, ctx->d_ssim_sums,
                    ctx->d_idx_all, ctx->d_sig_part, ctx->d_sig_count};
    for (void *p : bufs) if (p) cudaFree(p);
    if (ctx->ev_counts) {
        cudaEventSynchronize(ctx->ev_counts);  // no copy into h_totals may be left in flight
        cudaEventDestroy(ctx->ev_counts);
    }
    if (ctx->h_totals) cudaFreeHost(ctx->h_totals);
    for (auto &m : ctx->marks) { cudaEventDestroy(m.a); cudaEventDestroy(m.b); }
    for (cudaEvent_t e : ctx->event_pool) cudaEventDestroy(e);
    delete ctx;
    return SPARSEOIT_OK;
}

// set_active and set_active_async: `wait` selects whether the host waits for the counts now.
static int set_active_impl(sparseoit_ctx *ctx, const uint8_t *d_mask, int64_t n, void *stream, bool wait) {
    if (!ctx) return SPARSEOIT_ERR_INVALID_ARG;
    {
        const int rc = sync_counts(ctx);  // h_totals is about to be overwritten
        if (rc) return rc;
    }
    if (!d_mask && n > 0) return fail(ctx, SPARSEOIT_ERR_INVALID_ARG, "mask is null");
    if (n != ctx->N) return fail(ctx, SPARSEOIT_ERR_INVALID_ARG, "mask length differs from max_splats");
    cudaStream_t st = (cudaStream_t)stream;
    const uint8_t *prev = ctx->have_mask ? ctx->d_mask[ctx->cur] : nullptr;
    uint8_t *store = ctx->d_mask[ctx->cur ^ 1];
    {
        ProfScope ps(ctx, "compact", st);
        launch_compact(d_mask, prev, n, ctx->d_blk, ctx->d_totals, ctx->d_idx_active, ctx->d_idx_comp,
                       ctx->d_idx_plus, ctx->d_idx_minus, store, st);
    }
    CK_LAUNCH("compaction kernels");
    CK(cudaMemcpyAsync(ctx->h_totals, ctx->d_totals, 4 * sizeof(int64_t), cudaMemcpyDeviceToHost, st),
       "copy active counts");
    if (wait) {
        CK(cudaStreamSynchronize(st), "set_active sync");
        ctx->n_active = ctx->h_totals[0];
        ctx->n_comp = ctx->h_totals[1];
        ctx->n_plus = ctx->h_totals[2];
        ctx->n_minus = ctx->h_totals[3];
    } else {
        CK(cudaEventRecord(ctx->ev_counts, st), "record the active-count copy");
        ctx->counts_pending = true;
    }
    ctx->cur ^= 1;
    ctx->have_mask = true;
    ctx->generation += 1;
    ctx->have_fwd = false;
    return SPARSEOIT_OK;
}

int sparseoit_set_active(sparseoit_ctx *ctx, const uint8_t *d_mask, int64_t n, void *stream) {
    NvtxRange nvtx__("sparseoit_set_active");
    return set_active_impl(ctx, d_mask, n, stream, true);
}

int sparseoit_set_active_async(sparseoit_ctx *ctx, const uint8_t *d_mask, int64_t n, void *stream) {
    NvtxRange nvtx__("sparseoit_set_active_async");
    return set_active_impl(ctx, d_mask, n, stream, false);
}

int sparseoit_get_active(sparseoit_ctx *ctx, const int32_t **d_idx, int64_t *n_active) {
    if (!ctx || !d_idx || !n_active) return SPARSEOIT_ERR_INVALID_ARG;
    if (!ctx->have_mask) return fail(ctx, SPARSEOIT_ERR_STATE, "no active set yet");
    {
        const int rc = sync_counts(ctx);
        if (rc) return rc;
    }
    *d_idx = ctx->d_idx_active;
    *n_active = ctx->n_active;
    return SPARSEOIT_OK;
}

int sparseoit_get_frozen(sparseoit_ctx *ctx, int32_t view, float **d_planes) {
    if (!ctx || !d_planes) return SPARSEOIT_ERR_INVALID_ARG;
    if (view < 0 || view >= ctx->n_views) return fail(ctx, SPARSEOIT_ERR_INVALID_ARG, "view index out of range");
    *d_planes = ctx->d_frozen[view];
    return SPARSEOIT_OK;
}

int sparseoit_set_frozen(sparseoit_ctx *ctx, int32_t view, const float *planes, void *stream) {
    NvtxRange nvtx__("sparseoit_set_frozen");
    if (!ctx) return SPARSEOIT_ERR_INVALID_ARG;
    if (!planes) return fail(ctx, SPARSEOIT_ERR_INVALID_ARG, "null frozen planes");
    if (view < 0 || view >= ctx->n_views) return fail(ctx, SPARSEOIT_ERR_INVALID_ARG, "view index out of range");
    if (!ctx->have_mask) return fail(ctx, SPARSEOIT_ERR_STATE, "set_frozen before set_active");
    const size_t bytes = (size_t)5 * (size_t)ctx->W[view] * (size_t)ctx->H[view] * sizeof(float);
    CK(cudaMemcpyAsync(ctx->d_frozen[view], planes, bytes, cudaMemcpyDefault, (cudaStream_t)stream),
       "cudaMemcpyAsync(frozen planes)");
    ctx->view_gen[view] = ctx->generation;
    return SPARSEOIT_OK;
}

int sparseoit_commit_frozen(sparseoit_ctx *ctx, const sparseoit_splats *splats, const sparseoit_camera *cam,
                            int32_t view, int32_t mode, void *stream) {
    NvtxRange nvtx__("sparseoit_commit_frozen");
    if (!ctx) return SPARSEOIT_ERR_INVALID_ARG;
    int rc = check_splats(ctx, splats, false);
    if (rc) return rc;
    if (!ctx->have_mask) return fail(ctx, SPARSEOIT_ERR_STATE, "commit before set_active");
    if (mode != SPARSEOIT_COMMIT_INCREMENTAL && mode != SPARSEOIT_COMMIT_RECOMPUTE)
        return fail(ctx, SPARSEOIT_ERR_INVALID_ARG, "unknown commit mode");
    if (view < 0 || view >= ctx->n_views) return fail(ctx, SPARSEOIT_ERR_INVALID_ARG, "view index out of range");
    if (ctx->view_gen[view] == ctx->generation) return SPARSEOIT_OK;
    cudaStream_t st = (cudaStream_t)stream;
    Batch b;
    memset(&b, 0, sizeof(b));
    b.n_views = 1;
    rc = fill_view(ctx, cam, view, b.v[0], 0);
    if (rc) return rc;
    b.total_tiles = b.v[0].tiles_x * b.v[0].tiles_y;
    const bool incremental = mode == SPARSEOIT_COMMIT_INCREMENTAL && ctx->view_gen[view] == ctx->generation - 1;
    const int *l1, *l2 = nullptr;
    int64_t n1, n2 = 0;
    if (incremental) {
        l1 = ctx->d_idx_plus; n1 = ctx->n_plus;
        l2 = ctx->d_idx_minus; n2 = ctx->n_minus;
    } else {
        const int64_t hw = (int64_t)ctx->W[view] * ctx->H[view];
        CK(cudaMemsetAsync(ctx->d_frozen[view], 0, (size_t)(5 * hw) * sizeof(float), st), "memset(frozen)");
        l1 = ctx->d_idx_comp; n1 = ctx->n_comp;
    }
    b.n_list = (int)(n1 + n2);
    ctx->have_fwd = false;  // the commit reuses the forward's workspace
    if (b.n_list > 0) {
        rc = ensure_batch_ws(ctx, b.n_list, b.total_tiles);
        if (rc) return rc;
        rc = render_pass_bin(ctx, b, splats, l1, (int)n1, l2, (int)n2, st);
        if (rc) return rc;
        ProfScope ps(ctx, "raster_sums", st);
        launch_raster_fwd(b, kRasterSums, ctx->fwd_strip, ctx->d_rec, ctx->d_offsets, ctx->d_pairs, ctx->pair_cap,
                          splats->bg, nullptr, nullptr, ctx->fwd_persistent ? ctx->d_queue : nullptr, false, st);
        CK_LAUNCH("raster_fwd_kernel(sums)");
    }
    ctx->view_gen[view] = ctx->generation;
    return SPARSEOIT_OK;
}

// The forward over an index list: the context's active list composed with each view's frozen sums,
// or (whole_set) every splat of the scene with no frozen sums -- the full-set render of the
// active-set update, which leaves the active set and the frozen sums as they are.
static int forward_impl(sparseoit_ctx *ctx, const sparseoit_splats *splats, const sparseoit_camera *cams,
                        const int32_t *views, int32_t n_views, float *const *d_images, const float *const *d_targets,
                        float *d_loss, void *stream, bool whole_set) {
    if (!ctx) return SPARSEOIT_ERR_INVALID_ARG;
    int rc = check_splats(ctx, splats, !whole_set);
    if (rc) return rc;
    if (!whole_set && !ctx->have_mask) return fail(ctx, SPARSEOIT_ERR_STATE, "forward before set_active");
    if (n_views < 1 || n_views > kMaxViews || !cams || !views || !d_images)
        return fail(ctx, SPARSEOIT_ERR_INVALID_ARG, "bad view list");
    if (d_targets && !d_loss) return fail(ctx, SPARSEOIT_ERR_INVALID_ARG, "targets given without a loss pointer");
    cudaStream_t st = (cudaStream_t)stream;
    const int *list = ctx->d_idx_active;
    int64_t n_list = ctx->n_active;
    if (whole_set) {
        if (!ctx->d_idx_all) {
            std::vector<int> iota((size_t)ctx->N);
            for (int64_t i = 0; i < ctx->N; ++i) iota[(size_t)i] = (int)i;
            CK(cudaMalloc((void **)&ctx->d_idx_all, (size_t)ctx->N * sizeof(int)), "cudaMalloc(identity list)");
            CK(cudaMemcpy(ctx->d_idx_all, iota.data(), (size_t)ctx->N * sizeof(int), cudaMemcpyHostToDevice),
               "copy(identity list)");
        }
        list = ctx->d_idx_all;
        n_list = ctx->N;
    }
    Batch b;
    memset(&b, 0, sizeof(b));
    b.n_views = n_views;
    int tiles = 0;
    for (int k = 0; k < n_views; ++k) {
        const int v = views[k];
        if (v < 0 || v >= ctx->n_views) return fail(ctx, SPARSEOIT_ERR_INVALID_ARG, "view index out of range");
        for (int j = 0; j < k; ++j)
            if (views[j] == v) return fail(ctx, SPARSEOIT_ERR_INVALID_ARG, "a view is listed twice");
        if (!whole_set && ctx->view_gen[v] != ctx->generation)
            return fail(ctx, SPARSEOIT_ERR_STATE, "frozen sums of view " + std::to_string(v) +
                                                      " are stale: call sparseoit_commit_frozen first");
        rc = fill_view(ctx, &cams[k], v, b.v[k], tiles);
        if (rc) return rc;
        if (whole_set) b.v[k].frozen = nullptr;
        if (!d_images[k]) return fail(ctx, SPARSEOIT_ERR_INVALID_ARG, "image pointer is null");
        b.v[k].image = d_images[k];
        if (d_targets) {
            if (!d_targets[k]) return fail(ctx, SPARSEOIT_ERR_INVALID_ARG, "target pointer is null");
            b.v[k].target = d_targets[k];
        }
        tiles += b.v[k].tiles_x * b.v[k].tiles_y;
    }
    b.total_tiles = tiles;
    b.n_list = (int)n_list;
    while ((int)ctx->d_state.size() < n_views) ctx->d_state.push_back(nullptr);
    for (int k = 0; k < n_views; ++k) {
        if (!ctx->d_state[k]) CK(cudaMalloc((void **)&ctx->d_state[k], (size_t)(5 * ctx->max_pix) * sizeof(float)),
                                 "cudaMalloc(pixel state)");
        b.v[k].state = ctx->d_state[k];
    }
    rc = ensure_batch_ws(ctx, (int64_t)n_views * n_list, tiles);
    if (rc) return rc;
    if (d_loss) CK(cudaMemsetAsync(d_loss, 0, sizeof(float), st), "memset(loss)");
    if (ctx->counting) CK(cudaMemsetAsync(ctx->d_contrib, 0, sizeof(unsigned long long), st), "memset(counter)");
    // the backward's screen-space gradient sums, zeroed by the projection (no memset between the
    // forward raster and the backward raster)
    const int64_t nrec = (int64_t)n_views * n_list;
    CK(grow(&ctx->d_sgrad, &ctx->sgrad_cap, 3 * nrec), "cudaMalloc(screen grads)");
    ctx->sgrad_clean = false;
    rc = render_pass_bin(ctx, b, splats, list, (int)n_list, nullptr, 0, st, ctx->d_sgrad);
    if (rc) return rc;
    {
        ProfScope ps(ctx, "raster_fwd", st);
        launch_raster_fwd(b, d_targets ? kRasterFused : kRasterAux, ctx->fwd_strip, ctx->d_rec, ctx->d_offsets, ctx->d_pairs,
                          ctx->pair_cap, splats->bg, d_targets ? d_loss : nullptr,
                          ctx->counting ? ctx->d_contrib : nullptr, ctx->fwd_persistent ? ctx->d_queue : nullptr,
                          false, st);
    }
    CK_LAUNCH("raster_fwd_kernel");
    ctx->sgrad_clean = true;
    ctx->have_fwd = true;
    ctx->last_fused = d_targets != nullptr;
    ctx->planes_consumed = false;
    ctx->last_batch = b;
    ctx->last_list = list;
    ctx->last_n_list = (int)n_list;
    ctx->last_generation = ctx->generation;
    return SPARSEOIT_OK;
}

int sparseoit_forward(sparseoit_ctx *ctx, const sparseoit_splats *splats, const sparseoit_camera *cams,
                      const int32_t *views, int32_t n_views, float *const *d_images, const float *const *d_targets,
                      float *d_loss, void *stream) {
    NvtxRange nvtx__("sparseoit_forward");
    return forward_impl(ctx, splats, cams, views, n_views, d_images, d_targets, d_loss, stream, false);
}

int sparseoit_backward(sparseoit_ctx *ctx, const sparseoit_splats *splats, const float *const *d_grad_images,
                       sparseoit_grads *out, void *stream) {
    NvtxRange nvtx__("sparseoit_backward");
    if (!ctx) return SPARSEOIT_ERR_INVALID_ARG;
    int rc = check_splats(ctx, splats, true);
    if (rc) return rc;
    if (!ctx->have_fwd || ctx->last_generation != ctx->generation)
        return fail(ctx, SPARSEOIT_ERR_STATE, "backward without a matching forward");
    if (splats->rows == SPARSEOIT_ROWS_ACTIVE && ctx->last_list != ctx->d_idx_active)
        return fail(ctx, SPARSEOIT_ERR_INVALID_ARG, "active rows after a full-set forward");
    if (!out || !out->means || !out->quats || !out->log_scales || !out->opacity_logits || !out->sh_color ||
        !out->sh_weight || !out->sigma)
        return fail(ctx, SPARSEOIT_ERR_INVALID_ARG, "a gradient pointer is null");
    if (((uintptr_t)out->quats & 15u) || ((uintptr_t)out->sh_color & 15u) || ((uintptr_t)out->sh_weight & 15u))
        return fail(ctx, SPARSEOIT_ERR_INVALID_ARG, "quats / sh gradients must be 16-byte aligned");
    cudaStream_t st = (cudaStream_t)stream;
    Batch &b = ctx->last_batch;
    if (!ctx->last_fused) {
        if (ctx->planes_consumed)
            return fail(ctx, SPARSEOIT_ERR_STATE,
                        "backward: an earlier backward of this forward (no targets) consumed its planes; run the "
                        "forward again");
        if (!d_grad_images) return fail(ctx, SPARSEOIT_ERR_INVALID_ARG, "grad images needed (forward had no targets)");
        for (int k = 0; k < b.n_views; ++k) {
            if (!d_grad_images[k]) return fail(ctx, SPARSEOIT_ERR_INVALID_ARG, "grad image pointer is null");
            b.v[k].grad_image = d_grad_images[k];
        }
        ProfScope ps(ctx, "prep_state", st);
        launch_prep_state(b, splats->bg, st);
        CK_LAUNCH("prep_state_kernel");
        ctx->planes_consumed = true;
    }
    const int64_t nrec = (int64_t)b.n_views * ctx->last_n_list;
    // the forward's projection zeroed the screen-space sums; a second backward of the same forward
    // zeroes them here (and its raster then follows a memset: no programmatic launch)
    const bool clean = ctx->sgrad_clean && ctx->sgrad_cap >= 3 * nrec;
    if (!clean) {
        CK(grow(&ctx->d_sgrad, &ctx->sgrad_cap, 3 * nrec), "cudaMalloc(screen grads)");
        CK(cudaMemsetAsync(ctx->d_sgrad, 0, (size_t)(3 * nrec) * sizeof(float4), st), "memset(screen grads)");
    }
    ctx->sgrad_clean = false;
    const int chain_blocks = project_bwd_blocks(ctx->last_n_list);
    CK(grow(&ctx->d_sig_part, &ctx->sig_part_cap, chain_blocks > 0 ? chain_blocks : 1), "cudaMalloc(dsigma partials)");
    {
        ProfScope ps(ctx, "raster_bwd", st);
        if (ctx->bwd_parallel == 1)
            launch_raster_bwd(b, ctx->bwd_walk, ctx->d_rec, ctx->d_offsets, ctx->d_pairs, ctx->pair_cap,
                              ctx->d_sgrad, ctx->bwd_persistent ? ctx->d_queue + 1 : nullptr, clean && pdl_ok(ctx),
                              st);
        else
            launch_raster_bwd_pixel(b, ctx->bwd_parallel == 2, ctx->d_rec, ctx->d_offsets, ctx->d_pairs,
                                    ctx->pair_cap, ctx->d_sgrad, st);
    }
    CK_LAUNCH("raster_bwd_kernel");
    // dL/dsigma is written by the chain's last block; with no active splat there is no chain launch
    if (ctx->last_n_list == 0 && !out->accumulate)
        CK(cudaMemsetAsync(out->sigma, 0, sizeof(float), st), "memset(dsigma)");
    GradPtrs g{out->means,    out->quats,     out->log_scales,          out->opacity_logits,
               out->sh_color, out->sh_weight, out->sigma,               out->rows_by_splat != 0,
               out->accumulate != 0};
    {
        ProfScope ps(ctx, "project_bwd", st);
        launch_project_bwd(b, splat_ptrs(splats), splats->sh_dtype == SPARSEOIT_BF16, ctx->last_list,
                           ctx->last_n_list, ctx->d_sgrad, g, ctx->d_sig_part, ctx->d_sig_count, pdl_ok(ctx), st);
    }
    CK_LAUNCH("project_bwd_kernel");
    return SPARSEOIT_OK;
}

int sparseoit_update_active_set(sparseoit_ctx *ctx, const sparseoit_splats *splats, const sparseoit_camera *cams,
                                int32_t n_views, const float *const *d_targets, int32_t n_sub, int32_t first,
                                const float *eps, sparseoit_grads *scratch, uint8_t *d_mask, int32_t *sel_out,
                                void *stream) {
    NvtxRange nvtx__("sparseoit_update_active_set");
    if (!ctx) return SPARSEOIT_ERR_INVALID_ARG;
    if (!splats || !cams || !d_targets || !eps || !scratch || !d_mask)
        return fail(ctx, SPARSEOIT_ERR_INVALID_ARG, "update_active_set: null argument");
    if (n_views != ctx->n_views) return fail(ctx, SPARSEOIT_ERR_INVALID_ARG, "update_active_set: need every view");
    cudaStream_t st = (cudaStream_t)stream;
    std::vector<int32_t> sel(n_sub > 0 ? n_sub : 1);
    int rc = sparseoit_fps_views(cams, n_views, n_sub, first, sel.data());
    if (rc) return fail(ctx, rc, "update_active_set: bad view subsample (n_sub, first)");
    for (int k = 0; k < n_sub; ++k)
        if (!d_targets[sel[k]]) return fail(ctx, SPARSEOIT_ERR_INVALID_ARG, "update_active_set: null target");
    if (!ctx->d_upd_image) {
        CK(cudaMalloc((void **)&ctx->d_upd_image, (size_t)(3 * ctx->max_pix) * sizeof(float)), "cudaMalloc(update image)");
        CK(cudaMalloc((void **)&ctx->d_upd_loss, sizeof(float)), "cudaMalloc(update loss)");
    }
    // the full-set render of Alg. 1: every splat, no frozen sums, the current active set and the
    // views' frozen sums left as they are (so the commits after the update are incremental)
    sparseoit_grads g = *scratch;
    g.rows_by_splat = 1;
    for (int k = 0; k < n_sub; ++k) {
        const int32_t j = sel[k];
        float *img = ctx->d_upd_image;
        rc = forward_impl(ctx, splats, &cams[j], &j, 1, &img, &d_targets[j], ctx->d_upd_loss, stream, true);
        if (rc) return rc;
        g.accumulate = k > 0 ? 1 : 0;  // the gradient of the sum of the subsampled views' losses
        rc = sparseoit_backward(ctx, splats, nullptr, &g, stream);
        if (rc) return rc;
    }
    rc = sparseoit_activeness(&g, ctx->N, eps, d_mask, nullptr, stream);
    if (rc) return fail(ctx, rc, "update_active_set: activeness launch failed");
    rc = sparseoit_set_active(ctx, d_mask, ctx->N, stream);
    if (rc) return rc;
    if (sel_out)
        for (int k = 0; k < n_sub; ++k) sel_out[k] = sel[k];
    return SPARSEOIT_OK;
}

int sparseoit_adam_step(sparseoit_ctx *ctx, const sparseoit_grads *grads, sparseoit_rows *params, sparseoit_rows *m,
                        sparseoit_rows *v, const sparseoit_adam *cfg, void *stream) {
    NvtxRange nvtx__("sparseoit_adam_step");
    if (!ctx) return SPARSEOIT_ERR_INVALID_ARG;
    if (!grads || !params || !m || !v || !cfg) return fail(ctx, SPARSEOIT_ERR_INVALID_ARG, "adam: null argument");
    if (!ctx->have_mask) return fail(ctx, SPARSEOIT_ERR_STATE, "adam before set_active");
    {
        const int rc = sync_counts(ctx);
        if (rc) return rc;
    }
    if (cfg->step < 1 || !(cfg->beta1 >= 0.f && cfg->beta1 < 1.f) || !(cfg->beta2 >= 0.f && cfg->beta2 < 1.f) ||
        !(cfg->eps > 0.f))
        return fail(ctx, SPARSEOIT_ERR_INVALID_ARG, "adam: need step >= 1, 0 <= beta < 1, eps > 0");
    const float *g6[6] = {grads->means, grads->quats, grads->log_scales, grads->opacity_logits, grads->sh_color,
                          grads->sh_weight};
    sparseoit_rows *sets[3] = {params, m, v};
    soit::AdamArgs a;
    memset(&a, 0, sizeof(a));
    const int width[6] = {3, 4, 3, 1, 48, 16};
    for (int k = 0; k < 6; ++k) {
        float *row[3];
        for (int j = 0; j < 3; ++j) {
            sparseoit_rows *r = sets[j];
            float *q[6] = {r->means, r->quats, r->log_scales, r->opacity_logits, r->sh_color, r->sh_weight};
            row[j] = q[k];
        }
        if ((!g6[k] && ctx->n_active > 0) || !row[0] || !row[1] || !row[2])
            return fail(ctx, SPARSEOIT_ERR_INVALID_ARG, "adam: null array");
        a.g[k] = g6[k];
        a.p[k] = row[0];
        a.m[k] = row[1];
        a.v[k] = row[2];
        a.width[k] = width[k];
    }
    const bool sig = params->sigma || m->sigma || v->sigma;
    if (sig && !(params->sigma && m->sigma && v->sigma && grads->sigma))
        return fail(ctx, SPARSEOIT_ERR_INVALID_ARG, "adam: sigma pointers must be all given or all null");
    const double bc1 = 1.0 - std::pow((double)cfg->beta1, (double)cfg->step);
    const double bc2 = 1.0 - std::pow((double)cfg->beta2, (double)cfg->step);
    for (int j = 0; j < 8; ++j) a.step_size[j] = (float)(cfg->lr[j] / bc1);
    a.inv_sqrt_bc2 = (float)(1.0 / std::sqrt(bc2));
    a.beta1 = cfg->beta1;
    a.beta2 = cfg->beta2;
    a.eps = cfg->eps;
    a.idx = ctx->d_idx_active;
    a.n_active = ctx->n_active;
    if (cfg->rows != SPARSEOIT_ROWS_BY_SPLAT && cfg->rows != SPARSEOIT_ROWS_ACTIVE)
        return fail(ctx, SPARSEOIT_ERR_INVALID_ARG, "adam: unknown rows layout");
    a.active_rows = cfg->rows == SPARSEOIT_ROWS_ACTIVE ? 1 : 0;
    if (sig) {
        a.sigma_g = grads->sigma;
        a.sigma_p = params->sigma;
        a.sigma_m = m->sigma;
        a.sigma_v = v->sigma;
    }
    cudaStream_t st = (cudaStream_t)stream;
    {
        ProfScope ps(ctx, "adam", st);
        soit::launch_adam(a, st);
    }
    CK_LAUNCH("adam_kernel");
    return SPARSEOIT_OK;
}

int sparseoit_loss_l1_dssim(sparseoit_ctx *ctx, const float *const *d_targets, float lambda, float *d_loss,
                            float *const *d_grad_images, const float *bg, void *stream) {
    NvtxRange nvtx__("sparseoit_loss_l1_dssim");
    if (!ctx) return SPARSEOIT_ERR_INVALID_ARG;
    if (!d_targets || !d_loss || !bg) return fail(ctx, SPARSEOIT_ERR_INVALID_ARG, "loss: null argument");
    if (!(lambda >= 0.f && lambda <= 1.f)) return fail(ctx, SPARSEOIT_ERR_INVALID_ARG, "loss: lambda outside [0, 1]");
    if (!ctx->have_fwd || ctx->last_generation != ctx->generation || ctx->last_fused || ctx->planes_consumed)
        return fail(ctx, SPARSEOIT_ERR_STATE, "loss: needs the state of a forward run without targets");
    cudaStream_t st = (cudaStream_t)stream;
    Batch &b = ctx->last_batch;
    for (int k = 0; k < b.n_views; ++k)
        if (!d_targets[k]) return fail(ctx, SPARSEOIT_ERR_INVALID_ARG, "loss: null target");
    if (!ctx->d_ssim_abc) {
        CK(cudaMalloc((void **)&ctx->d_ssim_abc, (size_t)(9 * ctx->max_pix) * sizeof(float)), "cudaMalloc(ssim)");
        CK(cudaMalloc((void **)&ctx->d_ssim_sums, (size_t)(2 * kMaxViews) * sizeof(double)), "cudaMalloc(ssim sums)");
    }
    CK(cudaMemsetAsync(ctx->d_ssim_sums, 0, (size_t)(2 * b.n_views) * sizeof(double), st), "memset(ssim sums)");
    soit::SsimWindow win;
    {
        double g[11], sum = 0.0;
        for (int k = 0; k < 11; ++k) {
            const double x = k - 5;
            g[k] = std::exp(-x * x / (2.0 * 1.5 * 1.5));
            sum += g[k];
        }
        for (int k = 0; k < 11; ++k) win.w[k] = (float)(g[k] / sum);
    }
    soit::SsimLossArgs la;
    memset(&la, 0, sizeof(la));
    la.n_views = b.n_views;
    la.lambda = lambda;
    for (int k = 0; k < b.n_views; ++k) {
        const ViewDesc &vd = b.v[k];
        la.inv_n[k] = 1.0 / (3.0 * (double)vd.W * (double)vd.H);
        ProfScope ps(ctx, "ssim", st);
        soit::launch_ssim_view(vd.image, d_targets[k], vd.W, vd.H, win, ctx->d_ssim_abc, ctx->d_ssim_sums + 2 * k,
                               lambda, bg, vd.state, d_grad_images ? d_grad_images[k] : nullptr, st);
        CK_LAUNCH("ssim kernels");
    }
    soit::launch_ssim_loss(ctx->d_ssim_sums, la, d_loss, st);
    CK_LAUNCH("ssim_loss_kernel");
    ctx->last_fused = true;  // the state planes now hold the backward state
    return SPARSEOIT_OK;
}

static int rows_copy(sparseoit_ctx *ctx, const sparseoit_rows *src, sparseoit_rows *dst, int32_t sh_dtype,
                     bool to_active, void *stream) {
    if (!ctx) return SPARSEOIT_ERR_INVALID_ARG;
    if (!src || !dst) return fail(ctx, SPARSEOIT_ERR_INVALID_ARG, "rows: null argument");
    if (!ctx->have_mask) return fail(ctx, SPARSEOIT_ERR_STATE, "rows: before set_active");
    {
        const int rc = sync_counts(ctx);
        if (rc) return rc;
    }
    if (sh_dtype != SPARSEOIT_F32 && sh_dtype != SPARSEOIT_BF16)
        return fail(ctx, SPARSEOIT_ERR_INVALID_ARG, "rows: unknown sh_dtype");
    const float *s6[6] = {src->means, src->quats, src->log_scales, src->opacity_logits, src->sh_color, src->sh_weight};
    float *d6[6] = {dst->means, dst->quats, dst->log_scales, dst->opacity_logits, dst->sh_color, dst->sh_weight};
    const int width[6] = {3, 4, 3, 1, 48, 16};
    for (int k = 0; k < 6; ++k)
        if (!s6[k] || !d6[k]) return fail(ctx, SPARSEOIT_ERR_INVALID_ARG, "rows: null array");
    cudaStream_t st = (cudaStream_t)stream;
    for (int k = 0; k < 6; ++k) {
        const int eb = (k >= 4 && sh_dtype == SPARSEOIT_BF16) ? 2 : 4;
        soit::launch_rows_copy(ctx->d_idx_active, ctx->n_active, width[k], s6[k], d6[k], eb, to_active, st);
        CK_LAUNCH("rows_copy_kernel");
    }
    return SPARSEOIT_OK;
}

int sparseoit_gather_active(sparseoit_ctx *ctx, const sparseoit_rows *full, sparseoit_rows *active, int32_t sh_dtype,
                            void *stream) {
    return rows_copy(ctx, full, active, sh_dtype, true, stream);
}

int sparseoit_scatter_active(sparseoit_ctx *ctx, const sparseoit_rows *active, sparseoit_rows *full, int32_t sh_dtype,
                             void *stream) {
    return rows_copy(ctx, active, full, sh_dtype, false, stream);
}

// A persistent raster is chosen only if it beats the one-block-per-tile launch by 2 %: it is preceded
// by a memset of its queue, which forgoes the programmatic launch of the backward raster, and its
// timing in isolation is within noise of the other on most workloads.
constexpr float kPersistentMargin = 0.98f;

int sparseoit_autotune(sparseoit_ctx *ctx, const sparseoit_splats *splats, const sparseoit_camera *cams,
                       const int32_t *views, int32_t n_views, float *const *d_images, const float *const *d_targets,
                       float *d_loss, int32_t reps, sparseoit_tuning *out, void *stream) {
    NvtxRange nvtx__("sparseoit_autotune");
    if (!ctx || !out) return SPARSEOIT_ERR_INVALID_ARG;
    if (reps < 1) reps = 3;
    cudaStream_t st = (cudaStream_t)stream;
    const int cand[3] = {1, 2, 4};
    memset(out, 0, sizeof(*out));
    const bool prof = ctx->profiling;
    ctx->profiling = false;
    auto fwd = [&]() { return sparseoit_forward(ctx, splats, cams, views, n_views, d_images, d_targets, d_loss, stream); };
    // (1) the forward strip, one block per tile; then the chosen strip as persistent blocks
    ctx->fwd_persistent = false;
    int best = ctx->fwd_strip;
    float best_ms = 0.f;
    int rc = SPARSEOIT_OK;
    for (int c = 0; c < 3 && rc == SPARSEOIT_OK; ++c) {
        ctx->fwd_strip = cand[c];
        float ms = 0.f;
        rc = time_runs(ctx, st, reps, fwd, &ms);
        if (rc) break;
        out->candidates[out->n_candidates] = cand[c];
        out->ms[out->n_candidates] = ms;
        out->n_candidates++;
        if (c == 0 || ms < best_ms) { best_ms = ms; best = cand[c]; }
    }
    ctx->fwd_strip = best;
    out->fwd_pixels_per_thread = best;
    if (!rc) {
        ctx->fwd_persistent = true;
        rc = time_runs(ctx, st, reps, fwd, &out->fwd_persistent_ms);
        ctx->fwd_persistent = !rc && out->fwd_persistent_ms < kPersistentMargin * best_ms;
        out->fwd_persistent = ctx->fwd_persistent ? 1 : 0;
    }
    // (2) the backward raster on the fused forward's pixel state
    if (!rc && d_targets) rc = fwd();
    if (!rc && d_targets) {
        Batch &b = ctx->last_batch;
        const int64_t nrec = (int64_t)b.n_views * ctx->last_n_list;
        CK(grow(&ctx->d_sgrad, &ctx->sgrad_cap, 3 * nrec), "cudaMalloc(screen grads)");
        const int walks[2] = {kBwdWalkSorted, kBwdWalkArena};
        float best_b = 0.f;
        for (int k = 0; k < 4 && !rc; ++k) {
            const int walk = walks[k & 1];
            const bool pers = k >= 2;
            auto bwd = [&]() {
                CK(cudaMemsetAsync(ctx->d_sgrad, 0, (size_t)(3 * nrec) * sizeof(float4), st), "memset(screen grads)");
                ctx->sgrad_clean = false;  // the trial backward leaves its sums there
                launch_raster_bwd(b, walk, ctx->d_rec, ctx->d_offsets, ctx->d_pairs, ctx->pair_cap, ctx->d_sgrad,
                                  pers ? ctx->d_queue + 1 : nullptr, /*pdl=*/false, st);
                return cuda_check(ctx, cudaGetLastError(), "raster_bwd_kernel");
            };
            rc = time_runs(ctx, st, reps, bwd, &out->bwd_ms[k]);
            const float eff = pers ? out->bwd_ms[k] / kPersistentMargin : out->bwd_ms[k];
            if (!rc && (k == 0 || eff < best_b)) {
                best_b = eff;
                out->bwd_walk = walk;
                out->bwd_persistent = pers ? 1 : 0;
            }
        }
        if (!rc) {
            ctx->bwd_walk = out->bwd_walk;
            ctx->bwd_persistent = out->bwd_persistent != 0;
        }
    }
    ctx->profiling = prof;
    if (rc) return rc;
    // leave valid outputs of the chosen configuration
    return fwd();
}

int sparseoit_reserve_pairs(sparseoit_ctx *ctx, int64_t max_pairs) {
    if (!ctx) return SPARSEOIT_ERR_INVALID_ARG;
    if (max_pairs <= ctx->pair_cap) return SPARSEOIT_OK;
    if (max_pairs > 0x7fffffffll) return fail(ctx, SPARSEOIT_ERR_INVALID_ARG, "max_pairs above 2^31 - 1");
    CK(cudaDeviceSynchronize(), "reserve sync");
    if (ctx->d_pairs) cudaFree(ctx->d_pairs);
    ctx->d_pairs = nullptr;
    ctx->pair_cap = 0;
    CK(cudaMalloc((void **)&ctx->d_pairs, (size_t)max_pairs * sizeof(uint32_t)), "cudaMalloc(pairs)");
    ctx->pair_cap = max_pairs;
    ctx->have_fwd = false;
    return SPARSEOIT_OK;
}

int sparseoit_inject_scan_stall(sparseoit_ctx *ctx, int32_t partition) {
    if (!ctx) return SPARSEOIT_ERR_INVALID_ARG;
    if (partition < 0) return fail(ctx, SPARSEOIT_ERR_INVALID_ARG, "partition must be >= 0");
    ctx->scan_withhold = partition;
    return SPARSEOIT_OK;
}

int sparseoit_status(sparseoit_ctx *ctx, void *stream) {
    if (!ctx) return SPARSEOIT_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    unsigned h = 0;
    CK(cudaMemcpyAsync(&h, ctx->d_status, sizeof(unsigned), cudaMemcpyDeviceToHost, st), "read status");
    CK(cudaStreamSynchronize(st), "status sync");
    CK(cudaMemsetAsync(ctx->d_status, 0, sizeof(unsigned), st), "clear status");
    CK(cudaStreamSynchronize(st), "status sync");
    if (h & kStatusCapacity) return fail(ctx, SPARSEOIT_ERR_CAPACITY, "pair arena overflow");
    if (h & kStatusTimeout) return fail(ctx, SPARSEOIT_ERR_TIMEOUT, "a device-side wait gave up");
    return SPARSEOIT_OK;
}

int sparseoit_last_counts(sparseoit_ctx *ctx, void *stream, int64_t *n_pairs, int64_t *n_contrib) {
    if (!ctx) return SPARSEOIT_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    int64_t hp = 0;
    unsigned long long hc = 0;
    CK(cudaMemcpyAsync(&hp, ctx->d_npairs, sizeof(int64_t), cudaMemcpyDeviceToHost, st), "read pair count");
    CK(cudaMemcpyAsync(&hc, ctx->d_contrib, sizeof(unsigned long long), cudaMemcpyDeviceToHost, st),
       "read contrib count");
    CK(cudaStreamSynchronize(st), "counts sync");
    if (n_pairs) *n_pairs = hp;
    if (n_contrib) *n_contrib = (int64_t)hc;
    return SPARSEOIT_OK;
}

int sparseoit_set_profiling(sparseoit_ctx *ctx, int32_t enable) {
    if (!ctx) return SPARSEOIT_ERR_INVALID_ARG;
    ctx->profiling = enable != 0;
    return SPARSEOIT_OK;
}

int sparseoit_get_profile(sparseoit_ctx *ctx, int32_t max_entries, sparseoit_kernel_time *out, int32_t *n_out) {
    if (!ctx || !n_out || (max_entries > 0 && !out)) return SPARSEOIT_ERR_INVALID_ARG;
    std::map<std::string, std::pair<int64_t, double>> acc;
    for (auto &m : ctx->marks) {
        CK(cudaEventSynchronize(m.b), "profile sync");
        float ms = 0.f;
        CK(cudaEventElapsedTime(&ms, m.a, m.b), "profile elapsed");
        auto &e = acc[m.name];
        e.first += 1;
        e.second += ms;
        ctx->event_pool.push_back(m.a);
        ctx->event_pool.push_back(m.b);
    }
    ctx->marks.clear();
    int k = 0;
    for (auto &kv : acc) {
        if (k >= max_entries) break;
        memset(out[k].name, 0, sizeof(out[k].name));
        strncpy(out[k].name, kv.first.c_str(), sizeof(out[k].name) - 1);
        out[k].launches = kv.second.first;
        out[k].total_ms = kv.second.second;
        ++k;
    }
    *n_out = k;
    return SPARSEOIT_OK;
}

int sparseoit_set_counting(sparseoit_ctx *ctx, int32_t enable) {
    if (!ctx) return SPARSEOIT_ERR_INVALID_ARG;
    ctx->counting = enable != 0;
    return SPARSEOIT_OK;
}

}  // extern "C"
