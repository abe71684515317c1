// project.cu -- per-splat projection and SH evaluation (Eq. 1, 2, 4, 5, 6;
// Alg. 2 CullGaussian / ScreenspaceGaussians) and binning by tile id only
// (Alg. 2 CreateTiles / DuplicateWithKeys / SortByKeys / IdentifyTileRanges,
// App. A: "the sorting step only orders entries by tile ID").
//
// Binning is a counting sort: the projection counts, per tile, the splats
// whose cutoff ellipse {alpha_raw >= 1/255} meets the tile (exact per tile
// row, see row_tiles), one exclusive scan over the tiles of the batch
// gives the ranges, and a scatter pass appends each splat's record index to
// every tile it meets (a warp per splat).  The order inside a tile is
// arbitrary: Eq. 7 is a pair of sums and a product, independent of it.
#include "common.cuh"
#include "launch.h"

namespace soit {

// Tiles of view vd met by the ellipse
//     (A2 (dx - r dy))^2 + (B2 dy)^2 <= tau2,   (dx, dy) = pixel centre - (mx, my),
// e = (tau2, y half-extent, 1 / A2, dy at the rightmost point).
// tile_rows gives the tile rows [ty0, ty1]; row_tiles the tile columns
// [tx0, tx1] of one tile row.  For the band of pixel-centre rows of a tile
// row, the x-range of the ellipse is [mx + xl(dL), mx + xr(dR)] where
// xr(dy) = r dy + sqrt(tau2 - B2^2 dy^2)/A2 is concave and peaks at
// dy = dystar (xl convex, lowest at -dystar), so clamping the peak into the
// band gives the exact extent of each row.  All arithmetic is explicitly
// rounded: the count pass and the scatter pass evaluate these separately and
// must obtain identical tile sets.
__device__ __forceinline__ bool tile_rows(const ViewDesc &vd, float my, const float4 e, int &ty0, int &ty1) {
    const float tau2 = e.x, yh = e.y;
    if (!(tau2 > 0.f)) return false;
    const int py0 = f2i_clamped(ceilf(__fsub_rn(__fsub_rn(my, yh), 0.5f)), 0, vd.H);
    const int py1 = f2i_clamped(floorf(__fsub_rn(__fadd_rn(my, yh), 0.5f)), -1, vd.H - 1);
    if (py0 > py1) return false;
    ty0 = py0 / kTile;
    ty1 = py1 / kTile;
    return true;
}

// Square root by the PTX approximate instruction: deterministic for a given
// input, which is all the two passes need (the cutoff already carries a 2e-3
// relative margin for its error).
__device__ __forceinline__ float approx_sqrt(float x) {
    float y;
    asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

__device__ __forceinline__ bool row_tiles(const ViewDesc &vd, float mx, float my, float r, float B2,
                                          const float4 e, int ty, int &tx0, int &tx1) {
    const float tau2 = e.x, yh = e.y, invA2 = e.z, dys = e.w;
    const float ylo = fmaxf(__fsub_rn((float)(ty * kTile) + 0.5f, my), -yh);
    const float yhi = fminf(__fsub_rn((float)(ty * kTile + kTile - 1) + 0.5f, my), yh);
    if (ylo > yhi) return false;
    const float B2sq = __fmul_rn(B2, B2);
    const float dR = fminf(fmaxf(dys, ylo), yhi), dL = fminf(fmaxf(-dys, ylo), yhi);
    const float hR = __fmul_rn(approx_sqrt(fmaxf(__fsub_rn(tau2, __fmul_rn(B2sq, __fmul_rn(dR, dR))), 0.f)), invA2);
    const float hL = __fmul_rn(approx_sqrt(fmaxf(__fsub_rn(tau2, __fmul_rn(B2sq, __fmul_rn(dL, dL))), 0.f)), invA2);
    const float xr = __fadd_rn(mx, __fadd_rn(__fmul_rn(r, dR), hR));
    const float xl = __fadd_rn(mx, __fsub_rn(__fmul_rn(r, dL), hL));
    const int px0 = f2i_clamped(ceilf(__fsub_rn(xl, 0.501f)), 0, vd.W);
    const int px1 = f2i_clamped(floorf(__fsub_rn(xr, 0.499f)), -1, vd.W - 1);
    if (px0 > px1) return false;
    tx0 = px0 / kTile;
    tx1 = px1 / kTile;
    return true;
}

// G lanes (G = 1, 2, 4 or 16) per list entry r, looping over the views of the
// batch so that the splat's parameters are read from HBM once.  Lane k of the
// group loads the SH coefficients J k .. J k + J - 1 (J = 16 / G; one
// contiguous run, vector loads; the group reads the whole row), the
// lanes evaluate their basis values and sum the products with shuffles; the
// geometry is evaluated redundantly by the G lanes; the tile rows of the
// cutoff ellipse are counted by the lanes in parallel.  List entry r < n1 is
// splat list1[r] with sign +1, r >= n1 is splat list2[r - n1] with sign -1.
template <typename ShT, int G>
__global__ void __launch_bounds__(256, 3) project_kernel(const __grid_constant__ Batch b, SplatPtrs sp,
                                                      const int *__restrict__ list1, int n1,
                                                      const int *__restrict__ list2, int n2, float4 *__restrict__ rec,
                                                      float4 *__restrict__ ext, int *__restrict__ tile_count) {
    constexpr int J = 16 / G;
    const int r = (int)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) / G);  // uniform in a group
    const int k = threadIdx.x & (G - 1);
    const int n_list = n1 + n2;
    if (r >= n_list) return;  // whole groups leave together
    // parameter row: the splat's own row, or (active rows, forward only) the list entry itself
    const int i = sp.active_rows ? r : (r < n1 ? list1[r] : list2[r - n1]);
    const float sign = r < n1 ? 1.f : -1.f;

    float mu[3], q[4], ls[3];
    for (int j = 0; j < 3; ++j) mu[j] = __ldg(sp.means + 3 * (int64_t)i + j);
    const float4 q4 = __ldg(reinterpret_cast<const float4 *>(sp.quats) + i);
    q[0] = q4.x; q[1] = q4.y; q[2] = q4.z; q[3] = q4.w;
    for (int j = 0; j < 3; ++j) ls[j] = __ldg(sp.log_scales + 3 * (int64_t)i + j);
    const float ol = __ldg(sp.opacity_logits + i);
    // every load of the row is issued before the first arithmetic that waits on one
    const ShT *hc = reinterpret_cast<const ShT *>(sp.sh_color) + 48 * (int64_t)i;
    const ShT *hw = reinterpret_cast<const ShT *>(sp.sh_weight) + 16 * (int64_t)i;
    float h0[J], h1[J], h2[J], hv[J];
    load_sh_run<ShT, J>(hc, hw, J * k, h0, h1, h2, hv);
    const float o = 1.f / (1.f + expf(-ol));
    const float log2o = log2f(o);

    for (int v = 0; v < b.n_views; ++v) {
        const ViewDesc &vd = b.v[v];
        const int64_t qidx = (int64_t)v * n_list + r;
        float4 r0 = make_float4(0.f, 0.f, 0.f, 0.f), r1 = make_float4(0.f, -INFINITY, 0.f, -1.f);
        float4 r2 = make_float4(0.f, 0.f, 0.f, sign), e = make_float4(-1.f, 0.f, 0.f, 0.f);
        SplatGeom g;
        // the culling decision is uniform over the half-warp (same inputs, same code)
        if (o >= (1.f / 255.f) && splat_geometry(vd, mu, q, ls, g)) {
            const float z = g.tc[2], iz = 1.f / z;
            const float mx = fmaf(vd.fx, g.tc[0] * iz, vd.cx), my = fmaf(vd.fy, g.tc[1] * iz, vd.cy);
            const float rr = g.sxy / g.syy;
            const float A2 = sqrtf(kLog2e * g.syy / (2.f * g.det));
            const float B2 = sqrtf(kLog2e / (2.f * g.syy));
            // Eq. 4: SH colour and (Eq. 1) the single-channel weight SH
            const float idl = 1.f / g.dlen;
            float yk[J];
            sh_basis_group<G>(g.d[0] * idl, g.d[1] * idl, g.d[2] * idl, k, yk);
            float p0 = 0.f, p1 = 0.f, p2 = 0.f, pv = 0.f;
#pragma unroll
            for (int j = 0; j < J; ++j) {
                p0 = fmaf(yk[j], h0[j], p0);
                p1 = fmaf(yk[j], h1[j], p1);
                p2 = fmaf(yk[j], h2[j], p2);
                pv = fmaf(yk[j], hv[j], pv);
            }
            const unsigned gm = group_mask<G>();
            const float c0 = group_sum<G>(p0, gm) + 0.5f, c1 = group_sum<G>(p1, gm) + 0.5f;
            const float c2 = group_sum<G>(p2, gm) + 0.5f, vv = group_sum<G>(pv, gm) + 0.5f;
            const float w = fmaxf(0.f, 1.f - z / sp.sigma) * fmaxf(vv, 0.f);
            // cutoff: log2 alpha_raw >= -log2 255  <=>  quadratic <= log2(255 o);
            // widened slightly so that binning is a strict superset of the
            // pairs the raster accepts.
            const float tau = log2o + kLog2_255;
            if (tau > 0.f && isfinite(mx) && isfinite(my) && isfinite(A2) && isfinite(B2) && isfinite(rr) &&
                A2 > 0.f && B2 > 0.f) {
                const float tau2 = fmaf(tau, 2e-3f, tau) + 1e-3f;
                const float yh = sqrtf(tau2) / B2;
                const float xh = sqrtf(tau2 * fmaf(rr / B2, rr / B2, 1.f / (A2 * A2)));
                const float dys = tau2 * rr / (B2 * B2 * xh);
                r0 = make_float4(mx, my, rr, A2);
                r1 = make_float4(B2, log2o, w, yh);
                r2 = make_float4(fmaxf(c0, 0.f), fmaxf(c1, 0.f), fmaxf(c2, 0.f), sign);
                e = make_float4(tau2, yh, 1.f / A2, dys);
                int ty0, ty1;
                if (tile_rows(vd, my, e, ty0, ty1)) {
                    for (int ty = ty0 + k; ty <= ty1; ty += G) {
                        int tx0, tx1;
                        if (!row_tiles(vd, mx, my, rr, B2, e, ty, tx0, tx1)) continue;
                        int *row = tile_count + vd.tile_base + ty * vd.tiles_x;
                        for (int tx = tx0; tx <= tx1; ++tx) atomicAdd(row + tx, 1);
                    }
                }
            }
        }
        // the four 16-byte outputs, lane k of the group storing outputs k, k + G, ...
        if (G >= 4) {
            if (k == 0) rec[3 * qidx + 0] = r0;
            else if (k == 1) rec[3 * qidx + 1] = r1;
            else if (k == 2) rec[3 * qidx + 2] = r2;
            else if (k == 3) ext[qidx] = e;
        } else if (G == 2) {
            if (k == 0) {
                rec[3 * qidx + 0] = r0;
                rec[3 * qidx + 2] = r2;
            } else {
                rec[3 * qidx + 1] = r1;
                ext[qidx] = e;
            }
        } else {
            rec[3 * qidx + 0] = r0;
            rec[3 * qidx + 1] = r1;
            rec[3 * qidx + 2] = r2;
            ext[qidx] = e;
        }
    }
}

// Exclusive scan of the tile counts of the batch by one block of 1024
// threads, 8 consecutive counts per thread per chunk.  offsets[total] = M.
// cursor[t] = offsets[t] for the scatter.  Flags kStatusCapacity if M > cap.
// Load class of a tile with c pairs: 0 for an empty tile, else 1 + 4 e + m
// for c = 2^e (1 + m/4 + ...), i.e. four classes per octave (<= 124).
constexpr int kLoadClasses = 128;
__device__ __forceinline__ int load_class(int c) {
    if (c <= 0) return 0;
    const int e = 31 - __clz(c);
    const int m = (e >= 2 ? (c >> (e - 2)) : (c << (2 - e))) & 3;
    return 1 + 4 * e + m;
}

// One block: exclusive scan of the per-tile pair counts into offsets (and
// the scatter cursors), the capacity check, and, when order is given, the
// order in which the raster blocks take the tiles: by load class, heaviest
// first (a bucketed longest-processing-time-first schedule; the order
// within a class is arbitrary and changes no result).
__global__ void __launch_bounds__(1024) scan_tiles_kernel(const int *__restrict__ count, int total,
                                                          int *__restrict__ offsets, int *__restrict__ cursor,
                                                          int *__restrict__ order, int64_t cap, unsigned *status,
                                                          int64_t *pairs_out) {
    // one chunk of 8192 counts at a time, staged through shared memory so that the global loads
    // and stores are coalesced; element e sits at e + e / 32 (thread t's eight consecutive elements
    // then fall in distinct banks across the warp)
    __shared__ int sv[8192 + 8192 / 32];
    __shared__ int warp_sums[32];
    __shared__ int carry_s;
    __shared__ int cls_pos[kLoadClasses];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (tid == 0) carry_s = 0;
    __syncthreads();
    for (int base = 0; base < total; base += 1024 * 8) {
        const int nb = min(1024 * 8, total - base);
        for (int i = tid; i < 1024 * 8; i += 1024) sv[i + (i >> 5)] = i < nb ? count[base + i] : 0;
        __syncthreads();
        int vals[8];
        int local = 0;
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            const int e = tid * 8 + k;
            vals[k] = sv[e + (e >> 5)];
            local += vals[k];
        }
        int incl = local;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            int y = __shfl_up_sync(0xffffffffu, incl, off);
            if (lane >= off) incl += y;
        }
        if (lane == 31) warp_sums[warp] = incl;
        __syncthreads();
        if (warp == 0) {
            int ws = warp_sums[lane];
            int wi = ws;
#pragma unroll
            for (int off = 1; off < 32; off <<= 1) {
                int y = __shfl_up_sync(0xffffffffu, wi, off);
                if (lane >= off) wi += y;
            }
            warp_sums[lane] = wi - ws;  // exclusive
        }
        __syncthreads();
        const int carry = carry_s;
        int run = carry + warp_sums[warp] + incl - local;
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            const int e = tid * 8 + k;
            sv[e + (e >> 5)] = run;
            run += vals[k];
        }
        __syncthreads();
        for (int i = tid; i < nb; i += 1024) {
            const int o = sv[i + (i >> 5)];
            offsets[base + i] = o;
            cursor[base + i] = o;
        }
        if (tid == 1023) carry_s = run;
        __syncthreads();
    }
    if (tid == 0) {
        offsets[total] = carry_s;
        if (pairs_out) *pairs_out = carry_s;
        if ((int64_t)carry_s > cap) atomicOr(status, kStatusCapacity);
    }
    if (!order) return;
    for (int k = tid; k < kLoadClasses; k += 1024) cls_pos[k] = 0;
    __syncthreads();
    for (int i = tid; i < total; i += 1024) atomicAdd(&cls_pos[load_class(count[i])], 1);
    __syncthreads();
    if (warp == 0) {  // first position of each class, heaviest class first: a warp scan over
                      // the classes in descending order, four per lane
        int h[4], sum = 0;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            h[j] = cls_pos[kLoadClasses - 1 - (4 * lane + j)];
            sum += h[j];
        }
        int incl = sum;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, incl, off);
            if (lane >= off) incl += y;
        }
        int run = incl - sum;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            cls_pos[kLoadClasses - 1 - (4 * lane + j)] = run;
            run += h[j];
        }
    }
    __syncthreads();
    for (int i = tid; i < total; i += 1024) order[atomicAdd(&cls_pos[load_class(count[i])], 1)] = i;
}

// One warp per list entry.  Lanes compute the column range of one tile row
// each (32 rows at a time), a warp scan of the per-row counts flattens the
// entry's tile list, and each lane then takes one (row, column) of it, so a
// typical splat costs one round of position-returning atomics instead of one
// per row.
__global__ void __launch_bounds__(256, 8) scatter_kernel(const __grid_constant__ Batch b,
                                                         const float4 *__restrict__ rec,
                                                         const float4 *__restrict__ ext, int *__restrict__ cursor,
                                                         uint32_t *__restrict__ pairs, int64_t cap) {
    const int r = (int)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5);
    const int lane = threadIdx.x & 31;
    if (r >= b.n_list) return;  // whole warps leave together
    for (int v = 0; v < b.n_views; ++v) {
        const ViewDesc &vd = b.v[v];
        const int64_t qidx = (int64_t)v * b.n_list + r;
        // the three loads are issued together (the record is read even when the splat is culled)
        const float4 e = ext[qidx];
        const float4 r0 = rec[3 * qidx + 0];
        const float B2 = rec[3 * qidx + 1].x;
        int ty0, ty1;
        if (!(e.x > 0.f)) continue;
        if (!tile_rows(vd, r0.y, e, ty0, ty1)) continue;
        for (int tyb = ty0; tyb <= ty1; tyb += 32) {
            const int ty = tyb + lane;
            int tx0 = 0, cnt = 0;
            if (ty <= ty1) {
                int a0, a1;
                if (row_tiles(vd, r0.x, r0.y, r0.z, B2, e, ty, a0, a1)) {
                    tx0 = a0;
                    cnt = a1 - a0 + 1;
                }
            }
            int incl = cnt;  // inclusive scan of the per-row tile counts
#pragma unroll
            for (int off = 1; off < 32; off <<= 1) {
                const int y = __shfl_up_sync(0xffffffffu, incl, off);
                if (lane >= off) incl += y;
            }
            const int total = __shfl_sync(0xffffffffu, incl, 31);
            for (int base = 0; base < total; base += 32) {
                const int idx = base + lane;
                // row of flattened entry idx: the number of rows whose inclusive count is <= idx
                int row = 0;
#pragma unroll
                for (int step = 16; step > 0; step >>= 1) {
                    const int probe = __shfl_sync(0xffffffffu, incl, row + step - 1);
                    if (probe <= idx) row += step;
                }
                const int row_tx0 = __shfl_sync(0xffffffffu, tx0, row & 31);
                const int row_excl = __shfl_sync(0xffffffffu, incl - cnt, row & 31);
                if (idx < total) {
                    const int t = vd.tile_base + (tyb + row) * vd.tiles_x + row_tx0 + (idx - row_excl);
                    const int pos = atomicAdd(cursor + t, 1);
                    if ((int64_t)pos < cap) pairs[pos] = (uint32_t)qidx;
                }
            }
        }
    }
}

template <int G>
static void launch_project_g(const Batch &b, const SplatPtrs &sp, bool bf16, const int *list1, int n1,
                             const int *list2, int n2, float4 *rec, float4 *ext, int *tile_count, cudaStream_t st) {
    const int grid = (int)(((int64_t)(n1 + n2) * G + 255) / 256);
    if (bf16)
        project_kernel<__nv_bfloat16, G><<<grid, 256, 0, st>>>(b, sp, list1, n1, list2, n2, rec, ext, tile_count);
    else
        project_kernel<float, G><<<grid, 256, 0, st>>>(b, sp, list1, n1, list2, n2, rec, ext, tile_count);
}

int launch_project(const Batch &b, const SplatPtrs &sp, bool bf16, int lanes, const int *list1, int n1,
                   const int *list2, int n2, float4 *rec, float4 *ext, int *tile_count, cudaStream_t st) {
    if (n1 + n2 == 0) return 0;
    if (lanes == 16)
        launch_project_g<16>(b, sp, bf16, list1, n1, list2, n2, rec, ext, tile_count, st);
    else if (lanes == 2)
        launch_project_g<2>(b, sp, bf16, list1, n1, list2, n2, rec, ext, tile_count, st);
    else if (lanes == 1)
        launch_project_g<1>(b, sp, bf16, list1, n1, list2, n2, rec, ext, tile_count, st);
    else
        launch_project_g<4>(b, sp, bf16, list1, n1, list2, n2, rec, ext, tile_count, st);
    return 0;
}

int launch_scan_tiles(const int *count, int total, int *offsets, int *cursor, int *order, int64_t cap,
                      unsigned *status, int64_t *pairs_out, cudaStream_t st) {
    scan_tiles_kernel<<<1, 1024, 0, st>>>(count, total, offsets, cursor, order, cap, status, pairs_out);
    return 0;
}

int launch_scatter(const Batch &b, const float4 *rec, const float4 *ext, int *cursor, uint32_t *pairs, int64_t cap,
                   cudaStream_t st) {
    if (b.n_list == 0) return 0;
    scatter_kernel<<<(int)(((int64_t)b.n_list * 32 + 255) / 256), 256, 0, st>>>(b, rec, ext, cursor, pairs, cap);
    return 0;
}

}  // namespace soit
