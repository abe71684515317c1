// launch.h -- host-side launchers of the kernels (internal to libsparseoit).
#pragma once
#include <utility>

#include "common.cuh"

namespace soit {

// Launch `kernel` on `st`; pdl: with programmatic stream serialization, so that its blocks may start
// while the kernel enqueued just before it on `st` finishes (the kernel must call pdl_wait() before
// reading that kernel's outputs).  Use pdl only when the operation enqueued just before is a kernel.
template <typename... KArgs, typename... Args>
inline cudaError_t launch_kernel(void (*kernel)(KArgs...), dim3 grid, dim3 block, cudaStream_t st, bool pdl,
                                 Args &&...args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = 0;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = pdl ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}

// lanes = lanes per splat of the projection (4 or 16).  sgrad_zero (nullable): three float4 rows per
// record, zeroed for the backward raster's screen-space gradient sums.
int launch_project(const Batch &b, const SplatPtrs &sp, bool bf16, int lanes, const int *list1, int n1,
                   const int *list2, int n2, float4 *rec, float4 *ext, int *tile_count, float4 *sgrad_zero,
                   cudaStream_t st);
// sc: the zeroed scan scratch; withhold: partition that posts nothing (failure injection), else -1.
// pdl (here and below): launch with programmatic stream serialization (launch_kernel).
int launch_scan_tiles(const int *count, int total, int *offsets, int *cursor, ScanScratch sc, int64_t cap,
                      unsigned *status, int64_t *pairs_out, int withhold, bool pdl, cudaStream_t st);
// order (nullable): receives the raster blocks' tile order, heaviest load class first (placed by the
// scatter's first blocks from the scan's class histogram).
int launch_scatter(const Batch &b, const float4 *rec, const float4 *ext, int *cursor, uint32_t *pairs, int64_t cap,
                   const int *count, ScanScratch sc, int *order, bool pdl, cudaStream_t st);

enum RasterMode { kRasterFused = 0, kRasterAux = 1, kRasterSums = 2 };
// strip = pixels per thread of the forward raster (1, 2 or 4).
// queue (nullable): a zeroed-at-launch counter; given, the raster runs persistent blocks (as many as
// fit on the device) that take tiles from it in the raster order, else one block per tile.
int launch_raster_fwd(const Batch &b, int mode, int strip, const float4 *rec, const int *offsets,
                      const uint32_t *pairs, int64_t cap, const float bg[3], float *loss, unsigned long long *contrib,
                      int *queue, bool pdl, cudaStream_t st);

int launch_prep_state(const Batch &b, const float bg[3], cudaStream_t st);
// walk: kBwdWalkSorted (each tile's pairs sorted by first row before the warps take them) or
// kBwdWalkArena (arena order).
enum BwdWalk { kBwdWalkSorted = 1, kBwdWalkArena = 2 };
int launch_raster_bwd(const Batch &b, int walk, const float4 *rec, const int *offsets, const uint32_t *pairs,
                      int64_t cap, float4 *sgrad, int *queue, bool pdl, cudaStream_t st);

// Per-pixel backward (raster_bwd_pixel.cu), the ablation baseline: warp_reduce = sum the warp's
// pixels before the atomics, else one set of atomics per contributing pair.
int launch_raster_bwd_pixel(const Batch &b, bool warp_reduce, const float4 *rec, const int *offsets,
                            const uint32_t *pairs, int64_t cap, float4 *sgrad, cudaStream_t st);

struct GradPtrs {
    float *means, *quats, *log_scales, *opacity_logits, *sh_color, *sh_weight, *sigma;
    int rows_by_splat;
    int accumulate;
};
// sig_part: one float per block of the launch, sig_count: a counter that is zero at the launch (the
// last block to finish sums the blocks' dL/dsigma partials in block order and sets it back to zero).
int launch_project_bwd(const Batch &b, const SplatPtrs &sp, bool bf16, const int *list, int n, const float4 *sgrad,
                       GradPtrs out, float *sig_part, unsigned *sig_count, bool pdl, cudaStream_t st);
int project_bwd_blocks(int n);

int launch_compact(const uint8_t *mask_new, const uint8_t *mask_prev, int64_t n, int *blk_counts, int64_t *totals,
                   int *idx_active, int *idx_comp, int *idx_plus, int *idx_minus, uint8_t *mask_store,
                   cudaStream_t st);
int64_t compact_scratch_ints(int64_t n);

// Sparse Adam (adam.cu): group k = means, quats, log_scales, opacity, sh_color, sh_weight
// (blockIdx.y); step_size[j] = lr_j / (1 - beta1^t) for the 8 rate classes of sparseoit_adam.
struct AdamArgs {
    const int *idx;               // active index list [n_active]
    int64_t n_active;
    const float *g[6];            // compact gradient rows
    float *p[6], *m[6], *v[6];    // full rows by splat
    int width[6];
    float step_size[8];
    float inv_sqrt_bc2;           // 1 / sqrt(1 - beta2^t)
    float beta1, beta2, eps;
    const float *sigma_g;
    float *sigma_p, *sigma_m, *sigma_v;  // null: sigma not updated
    int active_rows;              // 1: p, m, v hold |A| rows in active order (like g)
};
int launch_adam(const AdamArgs &a, cudaStream_t st);
// Copy the active rows of one [N, w] array into [n_active, w] (to_active) or back; elem_bytes 4 or 2.
int launch_rows_copy(const int *idx, int64_t n_active, int w, const void *src, void *dst, int elem_bytes,
                     bool to_active, cudaStream_t st);

// D-SSIM loss (ssim.cu): the 11-tap Gaussian window, per-view loss constants.
struct SsimWindow {
    float w[11];
};
struct SsimLossArgs {
    int n_views;
    double lambda;
    double inv_n[kMaxViews];  // 1 / (3 H W) per view
};
// One view: abc = [3][H, W, 3] floats (scratch), sums = 2 doubles (S, |x - y|), state = the view's
// five planes (F, T, Q in; the backward state out), grad_out = dL/dC [H, W, 3] or null.
int launch_ssim_view(const float *img, const float *tgt, int W, int H, const SsimWindow &win, float *abc,
                     double *sums, float lambda, const float bg[3], float *state, float *grad_out, cudaStream_t st);
int launch_ssim_loss(const double *sums, const SsimLossArgs &a, float *loss, cudaStream_t st);

}  // namespace soit
