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
// e = (tau2, y half-extent, x half-extent, dy at the rightmost point).
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

__device__ __forceinline__ bool row_tiles(const ViewDesc &vd, float mx, float my, float r, float A2, float B2,
                                          const float4 e, int ty, int &tx0, int &tx1) {
    const float tau2 = e.x, yh = e.y, dys = e.w;
    const float ylo = fmaxf(__fsub_rn((float)(ty * kTile) + 0.5f, my), -yh);
    const float yhi = fminf(__fsub_rn((float)(ty * kTile + kTile - 1) + 0.5f, my), yh);
    if (ylo > yhi) return false;
    const float invA2 = __fdiv_rn(1.f, A2), B2sq = __fmul_rn(B2, B2);
    const float dR = fminf(fmaxf(dys, ylo), yhi), dL = fminf(fmaxf(-dys, ylo), yhi);
    const float hR = __fmul_rn(__fsqrt_rn(fmaxf(__fsub_rn(tau2, __fmul_rn(B2sq, __fmul_rn(dR, dR))), 0.f)), invA2);
    const float hL = __fmul_rn(__fsqrt_rn(fmaxf(__fsub_rn(tau2, __fmul_rn(B2sq, __fmul_rn(dL, dL))), 0.f)), invA2);
    const float xr = __fadd_rn(mx, __fadd_rn(__fmul_rn(r, dR), hR));
    const float xl = __fadd_rn(mx, __fsub_rn(__fmul_rn(r, dL), hL));
    const int px0 = f2i_clamped(ceilf(__fsub_rn(xl, 0.501f)), 0, vd.W);
    const int px1 = f2i_clamped(floorf(__fsub_rn(xr, 0.499f)), -1, vd.W - 1);
    if (px0 > px1) return false;
    tx0 = px0 / kTile;
    tx1 = px1 / kTile;
    return true;
}

// One thread per list entry r; loops over the views of the batch so that the
// splat's parameters are read from HBM once.  List entry r < n1 is splat
// list1[r] with sign +1, r >= n1 is splat list2[r - n1] with sign -1.
template <typename ShT>
__global__ void __launch_bounds__(256) project_kernel(const __grid_constant__ Batch b, SplatPtrs sp,
                                                      const int *__restrict__ list1, int n1,
                                                      const int *__restrict__ list2, int n2, float4 *__restrict__ rec,
                                                      float4 *__restrict__ ext, int *__restrict__ tile_count) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    const int n_list = n1 + n2;
    if (r >= n_list) return;
    const int i = r < n1 ? list1[r] : list2[r - n1];
    const float sign = r < n1 ? 1.f : -1.f;

    float mu[3], q[4], ls[3];
    for (int k = 0; k < 3; ++k) mu[k] = __ldg(sp.means + 3 * (int64_t)i + k);
    const float4 q4 = __ldg(reinterpret_cast<const float4 *>(sp.quats) + i);
    q[0] = q4.x; q[1] = q4.y; q[2] = q4.z; q[3] = q4.w;
    for (int k = 0; k < 3; ++k) ls[k] = __ldg(sp.log_scales + 3 * (int64_t)i + k);
    const float ol = __ldg(sp.opacity_logits + i);
    const float o = 1.f / (1.f + expf(-ol));
    const float log2o = log2f(o);
    const ShT *hc = reinterpret_cast<const ShT *>(sp.sh_color) + 48 * (int64_t)i;
    const ShT *hw = reinterpret_cast<const ShT *>(sp.sh_weight) + 16 * (int64_t)i;

    for (int v = 0; v < b.n_views; ++v) {
        const ViewDesc &vd = b.v[v];
        const int64_t qidx = (int64_t)v * n_list + r;
        float4 r0 = make_float4(0.f, 0.f, 0.f, 0.f), r1 = make_float4(0.f, -INFINITY, 0.f, 0.f);
        float4 r2 = make_float4(0.f, 0.f, 0.f, sign), e = make_float4(-1.f, 0.f, 0.f, 0.f);
        SplatGeom g;
        if (o >= (1.f / 255.f) && splat_geometry(vd, mu, q, ls, g)) {
            const float z = g.tc[2], iz = 1.f / z;
            const float mx = fmaf(vd.fx, g.tc[0] * iz, vd.cx), my = fmaf(vd.fy, g.tc[1] * iz, vd.cy);
            const float rr = g.sxy / g.syy;
            const float A2 = sqrtf(kLog2e * g.syy / (2.f * g.det));
            const float B2 = sqrtf(kLog2e / (2.f * g.syy));
            // Eq. 4: SH colour and (Eq. 1) the single-channel weight SH
            const float idl = 1.f / g.dlen;
            float Y[16];
            sh_basis16(g.d[0] * idl, g.d[1] * idl, g.d[2] * idl, Y);
            float c0 = 0.5f, c1 = 0.5f, c2 = 0.5f, vv = 0.5f;
#pragma unroll
            for (int k = 0; k < 16; ++k) {
                c0 = fmaf(Y[k], ldf(hc, 3 * k + 0), c0);
                c1 = fmaf(Y[k], ldf(hc, 3 * k + 1), c1);
                c2 = fmaf(Y[k], ldf(hc, 3 * k + 2), c2);
                vv = fmaf(Y[k], ldf(hw, k), vv);
            }
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
                e = make_float4(tau2, yh, xh, dys);
                int ty0, ty1;
                if (tile_rows(vd, my, e, ty0, ty1)) {
                    for (int ty = ty0; ty <= ty1; ++ty) {
                        int tx0, tx1;
                        if (!row_tiles(vd, mx, my, rr, A2, B2, e, ty, tx0, tx1)) continue;
                        int *row = tile_count + vd.tile_base + ty * vd.tiles_x;
                        for (int tx = tx0; tx <= tx1; ++tx) atomicAdd(row + tx, 1);
                    }
                }
            }
        }
        rec[3 * qidx + 0] = r0;
        rec[3 * qidx + 1] = r1;
        rec[3 * qidx + 2] = r2;
        ext[qidx] = e;
    }
}

// Exclusive scan of the tile counts of the batch by one block of 1024
// threads, 8 consecutive counts per thread per chunk.  offsets[total] = M.
// cursor[t] = offsets[t] for the scatter.  Flags kStatusCapacity if M > cap.
__global__ void __launch_bounds__(1024) scan_tiles_kernel(const int *__restrict__ count, int total,
                                                          int *__restrict__ offsets, int *__restrict__ cursor,
                                                          int64_t cap, unsigned *status, int64_t *pairs_out) {
    __shared__ int warp_sums[32];
    __shared__ int carry_s;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (tid == 0) carry_s = 0;
    __syncthreads();
    for (int base = 0; base < total; base += 1024 * 8) {
        int vals[8];
        int local = 0;
        const int i0 = base + tid * 8;
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            vals[k] = (i0 + k < total) ? count[i0 + k] : 0;
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
            if (i0 + k < total) {
                offsets[i0 + k] = run;
                cursor[i0 + k] = run;
            }
            run += vals[k];
        }
        __syncthreads();
        if (tid == 1023) carry_s = run;
        __syncthreads();
    }
    if (tid == 0) {
        offsets[total] = carry_s;
        if (pairs_out) *pairs_out = carry_s;
        if ((int64_t)carry_s > cap) atomicOr(status, kStatusCapacity);
    }
}

// One warp per list entry: the warp walks the entry's tile rows and its
// lanes take the columns of a row in parallel, so the position-returning
// atomics of a splat overlap instead of running one after another.
__global__ void __launch_bounds__(256) scatter_kernel(const __grid_constant__ Batch b, const float4 *__restrict__ rec,
                                                      const float4 *__restrict__ ext, int *__restrict__ cursor,
                                                      uint32_t *__restrict__ pairs, int64_t cap) {
    const int r = (int)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5);
    const int lane = threadIdx.x & 31;
    if (r >= b.n_list) return;
    for (int v = 0; v < b.n_views; ++v) {
        const ViewDesc &vd = b.v[v];
        const int64_t qidx = (int64_t)v * b.n_list + r;
        const float4 e = ext[qidx];
        int ty0, ty1;
        if (!(e.x > 0.f)) continue;
        const float4 r0 = rec[3 * qidx + 0];
        if (!tile_rows(vd, r0.y, e, ty0, ty1)) continue;
        const float B2 = rec[3 * qidx + 1].x;
        for (int ty = ty0; ty <= ty1; ++ty) {
            int tx0, tx1;
            if (!row_tiles(vd, r0.x, r0.y, r0.z, r0.w, B2, e, ty, tx0, tx1)) continue;
            int *row = cursor + vd.tile_base + ty * vd.tiles_x;
            for (int tx = tx0 + lane; tx <= tx1; tx += 32) {
                const int pos = atomicAdd(row + tx, 1);
                if ((int64_t)pos < cap) pairs[pos] = (uint32_t)qidx;
            }
        }
    }
}

int launch_project(const Batch &b, const SplatPtrs &sp, bool bf16, const int *list1, int n1, const int *list2, int n2,
                   float4 *rec, float4 *ext, int *tile_count, cudaStream_t st) {
    const int n = n1 + n2;
    if (n == 0) return 0;
    const int grid = (n + 255) / 256;
    if (bf16)
        project_kernel<__nv_bfloat16><<<grid, 256, 0, st>>>(b, sp, list1, n1, list2, n2, rec, ext, tile_count);
    else
        project_kernel<float><<<grid, 256, 0, st>>>(b, sp, list1, n1, list2, n2, rec, ext, tile_count);
    return 0;
}

int launch_scan_tiles(const int *count, int total, int *offsets, int *cursor, int64_t cap, unsigned *status,
                      int64_t *pairs_out, cudaStream_t st) {
    scan_tiles_kernel<<<1, 1024, 0, st>>>(count, total, offsets, cursor, cap, status, pairs_out);
    return 0;
}

int launch_scatter(const Batch &b, const float4 *rec, const float4 *ext, int *cursor, uint32_t *pairs, int64_t cap,
                   cudaStream_t st) {
    if (b.n_list == 0) return 0;
    scatter_kernel<<<(int)(((int64_t)b.n_list * 32 + 255) / 256), 256, 0, st>>>(b, rec, ext, cursor, pairs, cap);
    return 0;
}

}  // namespace soit
