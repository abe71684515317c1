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
                                                      float4 *__restrict__ ext, int *__restrict__ tile_count,
                                                      float4 *__restrict__ sgrad_zero) {
    constexpr int J = 16 / G;
    pdl_allow_next();  // launched after everything before it completed: the scan may become resident
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
                        int *row = tile_count + (int64_t)(vd.tile_base + ty * vd.tiles_x) * kTileCounterStride;
                        for (int tx = tx0; tx <= tx1; ++tx) atomicAdd(row + tx * kTileCounterStride, 1);
                    }
                }
            }
        }
        // the four 16-byte outputs, lane k of the group storing outputs k, k + G, ...; and the
        // record's three rows of screen-space gradient sums zeroed for the backward raster's atomics
        const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
        if (G >= 4) {
            if (k == 0) rec[3 * qidx + 0] = r0;
            else if (k == 1) rec[3 * qidx + 1] = r1;
            else if (k == 2) rec[3 * qidx + 2] = r2;
            else if (k == 3) ext[qidx] = e;
            if (sgrad_zero && k < 3) sgrad_zero[3 * qidx + k] = z4;
        } else if (G == 2) {
            if (k == 0) {
                rec[3 * qidx + 0] = r0;
                rec[3 * qidx + 2] = r2;
                if (sgrad_zero) sgrad_zero[3 * qidx + 0] = sgrad_zero[3 * qidx + 2] = z4;
            } else {
                rec[3 * qidx + 1] = r1;
                ext[qidx] = e;
                if (sgrad_zero) sgrad_zero[3 * qidx + 1] = z4;
            }
        } else {
            rec[3 * qidx + 0] = r0;
            rec[3 * qidx + 1] = r1;
            rec[3 * qidx + 2] = r2;
            ext[qidx] = e;
            if (sgrad_zero) sgrad_zero[3 * qidx + 0] = sgrad_zero[3 * qidx + 1] = sgrad_zero[3 * qidx + 2] = z4;
        }
    }
}

// Load class of a tile with c pairs: 0 for an empty tile, else 1 + 4 e + m
// for c = 2^e (1 + m/4 + ...), i.e. four classes per octave (<= 124).
__device__ __forceinline__ int load_class(int c) {
    if (c <= 0) return 0;
    const int e = 31 - __clz(c);
    const int m = (e >= 2 ? (c >> (e - 2)) : (c << (2 - e))) & 3;
    return 1 + 4 * e + m;
}

// %globaltimer (nanoseconds) for the deadline of a bounded wait.
__device__ __forceinline__ uint64_t global_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Partition state words of the look-back scan: flag in the top two bits, value below.
constexpr unsigned long long kPartAgg = 1ull << 62, kPartPrefix = 2ull << 62, kPartValue = (1ull << 62) - 1;
constexpr unsigned long long kScanWaitNs = 250000000ull;  // a partition gives up waiting after 0.25 s

// Exclusive scan of the batch's per-tile pair counts into offsets (and the
// scatter cursors) in one pass over kScanItems-tile partitions, by decoupled
// look-back: a block takes the next partition number from a ticket counter
// (so that every lower partition belongs to a block that is already running),
// scans its counts, posts its aggregate, then walks back over the lower
// partitions' posts until it meets an inclusive prefix, and posts its own.
// Each wait for a post is bounded: after kScanWaitNs the block sets
// kStatusTimeout, writes nothing and returns (the kernels after it see the
// status word and skip their work).  The last partition writes offsets[total]
// = M and flags kStatusCapacity if M exceeds the pair arena.  Each block also
// adds its tiles' load classes into the batch's class histogram.
// `withhold`: the partition that posts nothing (failure injection for tests;
// -1 in normal use).
__global__ void __launch_bounds__(kScanThreads) scan_tiles_kernel(const int *__restrict__ count, int total,
                                                                  int *__restrict__ offsets,
                                                                  int *__restrict__ cursor, ScanScratch sc,
                                                                  int64_t cap, unsigned *status, int64_t *pairs_out,
                                                                  int withhold) {
    __shared__ int part_s, warp_sums[kScanThreads / 32];
    __shared__ long long excl_s;
    __shared__ int bad_s;
    __shared__ int cls[kLoadClasses];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    pdl_wait();  // the projection's tile counts
    pdl_allow_next();
    if (tid == 0) part_s = atomicAdd(sc.ticket, 1);
    for (int k = tid; k < kLoadClasses; k += kScanThreads) cls[k] = 0;
    __syncthreads();
    const int part = part_s;
    const int base = part * kScanItems + tid * kScanPer;
    int v[kScanPer], local = 0;
#pragma unroll
    for (int k = 0; k < kScanPer; ++k) {
        v[k] = base + k < total ? count[(int64_t)(base + k) * kTileCounterStride] : 0;
        local += v[k];
        if (base + k < total) atomicAdd(&cls[load_class(v[k])], 1);
    }
    int incl = local;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, incl, off);
        if (lane >= off) incl += y;
    }
    if (lane == 31) warp_sums[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        const int ws = lane < kScanThreads / 32 ? warp_sums[lane] : 0;
        int wi = ws;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, wi, off);
            if (lane >= off) wi += y;
        }
        if (lane < kScanThreads / 32) warp_sums[lane] = wi - ws;  // exclusive
        if (lane == kScanThreads / 32 - 1) {                      // this thread holds the aggregate
            const unsigned long long agg = (unsigned long long)wi;
            unsigned long long *state = sc.state;
            long long excl = 0;
            int bad = 0;
            if (part != withhold) atomicExch(state + part, (part == 0 ? kPartPrefix : kPartAgg) | agg);
            if (part > 0) {
                const uint64_t deadline = global_ns() + kScanWaitNs;
                for (int j = part - 1; j >= 0;) {
                    const unsigned long long w = *(volatile unsigned long long *)(state + j);
                    if ((w & ~kPartValue) == 0) {  // not posted yet
                        if (global_ns() > deadline) {
                            bad = 1;
                            break;
                        }
                        __nanosleep(64);
                        continue;
                    }
                    excl += (long long)(w & kPartValue);
                    if (w & kPartPrefix) break;
                    --j;
                }
                if (!bad && part != withhold)
                    atomicExch(state + part, kPartPrefix | (unsigned long long)(excl + (long long)agg));
            }
            if (bad) atomicOr(status, kStatusTimeout);
            excl_s = excl;
            bad_s = bad;
            if (!bad && (int64_t)(part + 1) * kScanItems >= total) {  // the last partition
                const long long M = excl + (long long)agg;
                offsets[total] = (int)M;
                if (pairs_out) *pairs_out = M;
                if (M > cap) atomicOr(status, kStatusCapacity);
            }
        }
    }
    __syncthreads();
    if (bad_s) return;
    int run = (int)excl_s + warp_sums[warp] + incl - local;
#pragma unroll
    for (int k = 0; k < kScanPer; ++k) {
        if (base + k < total) {
            offsets[base + k] = run;
            cursor[base + k] = run;
        }
        run += v[k];
    }
    for (int k = tid; k < kLoadClasses; k += kScanThreads)
        if (cls[k]) atomicAdd(sc.class_hist + k, cls[k]);
}

// The raster blocks' tile order: by load class, heaviest first (a bucketed
// longest-processing-time-first schedule; the order within a class is
// arbitrary and changes no result).  Block `blk` places tiles
// [256 blk, 256 blk + 256): it derives the classes' first positions from the
// batch's class histogram, reserves one range per class for its tiles with
// one atomic, and places them.  Run by the first blocks of the scatter (the
// scan is complete by then).
__device__ __forceinline__ void place_tile_order(const int *__restrict__ count, int total, const ScanScratch &sc,
                                                 int *__restrict__ order, int blk) {
    __shared__ int first[kLoadClasses], local[kLoadClasses], base_s[kLoadClasses];
    const int tid = threadIdx.x, lane = tid & 31;
    for (int k = tid; k < kLoadClasses; k += kScanThreads) local[k] = 0;
    if (tid < 32) {  // descending exclusive scan of the class histogram, four classes per lane
        int h[4], sum = 0;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            h[j] = sc.class_hist[kLoadClasses - 1 - (4 * lane + j)];
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
            first[kLoadClasses - 1 - (4 * lane + j)] = run;
            run += h[j];
        }
    }
    __syncthreads();
    const int t = blk * kScanThreads + tid;
    int c = 0, slot = 0;
    if (t < total) {
        c = load_class(count[(int64_t)t * kTileCounterStride]);
        slot = atomicAdd(&local[c], 1);
    }
    __syncthreads();
    for (int k = tid; k < kLoadClasses; k += kScanThreads)
        if (local[k]) base_s[k] = first[k] + atomicAdd(sc.class_cursor + k, local[k]);
    __syncthreads();
    if (t < total) order[base_s[c] + slot] = t;
}

// One warp per list entry.  Lanes compute the column range of one tile row
// each (32 rows at a time), a warp scan of the per-row counts flattens the
// entry's tile list, and each lane then takes one (row, column) of it, so a
// typical splat costs one round of position-returning atomics instead of one
// per row.
// The first order_blocks blocks (256 threads) also place the raster tile order (place_tile_order).
__global__ void __launch_bounds__(256, 8) scatter_kernel(const __grid_constant__ Batch b,
                                                         const float4 *__restrict__ rec,
                                                         const float4 *__restrict__ ext, int *__restrict__ cursor,
                                                         uint32_t *__restrict__ pairs, int64_t cap,
                                                         const int *__restrict__ count, ScanScratch sc, int *order,
                                                         int order_blocks) {
    const int r = (int)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5);
    const int lane = threadIdx.x & 31;
    // the first view's record, written by the projection (complete before the scan got past its own
    // wait), is read while the scan may still be running
    float4 e = make_float4(-1.f, 0.f, 0.f, 0.f), r0 = e;
    float B2 = 0.f;
    if (r < b.n_list) {
        e = ext[r];
        r0 = rec[3 * (int64_t)r + 0];
        B2 = rec[3 * (int64_t)r + 1].x;
    }
    pdl_wait();  // the scan's offsets, cursors, class histogram and status
    pdl_allow_next();
    if ((int)blockIdx.x < order_blocks && !bin_failed(b)) place_tile_order(count, b.total_tiles, sc, order, blockIdx.x);
    if (r >= b.n_list) return;  // whole warps leave together
    for (int v = 0; v < b.n_views; ++v) {
        const ViewDesc &vd = b.v[v];
        const int64_t qidx = (int64_t)v * b.n_list + r;
        if (v > 0) {  // the loads are issued together (the record is read even when the splat is culled)
            e = ext[qidx];
            r0 = rec[3 * qidx + 0];
            B2 = rec[3 * qidx + 1].x;
        }
        // if the tile scan gave up, its offsets are incomplete
        const unsigned stat = __ldg(b.status);
        int ty0, ty1;
        if (stat & kStatusTimeout) return;
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
                             const int *list2, int n2, float4 *rec, float4 *ext, int *tile_count, float4 *sgrad_zero,
                             cudaStream_t st) {
    const int grid = (int)(((int64_t)(n1 + n2) * G + 255) / 256);
    if (bf16)
        project_kernel<__nv_bfloat16, G>
            <<<grid, 256, 0, st>>>(b, sp, list1, n1, list2, n2, rec, ext, tile_count, sgrad_zero);
    else
        project_kernel<float, G><<<grid, 256, 0, st>>>(b, sp, list1, n1, list2, n2, rec, ext, tile_count, sgrad_zero);
}

int launch_project(const Batch &b, const SplatPtrs &sp, bool bf16, int lanes, const int *list1, int n1,
                   const int *list2, int n2, float4 *rec, float4 *ext, int *tile_count, float4 *sgrad_zero,
                   cudaStream_t st) {
    if (n1 + n2 == 0) return 0;
    if (lanes == 16)
        launch_project_g<16>(b, sp, bf16, list1, n1, list2, n2, rec, ext, tile_count, sgrad_zero, st);
    else if (lanes == 2)
        launch_project_g<2>(b, sp, bf16, list1, n1, list2, n2, rec, ext, tile_count, sgrad_zero, st);
    else if (lanes == 1)
        launch_project_g<1>(b, sp, bf16, list1, n1, list2, n2, rec, ext, tile_count, sgrad_zero, st);
    else
        launch_project_g<4>(b, sp, bf16, list1, n1, list2, n2, rec, ext, tile_count, sgrad_zero, st);
    return 0;
}

int launch_scan_tiles(const int *count, int total, int *offsets, int *cursor, ScanScratch sc, int64_t cap,
                      unsigned *status, int64_t *pairs_out, int withhold, bool pdl, cudaStream_t st) {
    launch_kernel(scan_tiles_kernel, dim3(scan_partitions(total)), dim3(kScanThreads), st, pdl, count, total, offsets,
                  cursor, sc, cap, status, pairs_out, withhold);
    return 0;
}

int launch_scatter(const Batch &b, const float4 *rec, const float4 *ext, int *cursor, uint32_t *pairs, int64_t cap,
                   const int *count, ScanScratch sc, int *order, bool pdl, cudaStream_t st) {
    const int order_blocks = order ? (b.total_tiles + kScanThreads - 1) / kScanThreads : 0;
    const int scatter_blocks = (int)(((int64_t)b.n_list * 32 + 255) / 256);
    const int grid = scatter_blocks > order_blocks ? scatter_blocks : order_blocks;
    if (grid == 0) return 0;
    launch_kernel(scatter_kernel, dim3(grid), dim3(256), st, pdl, b, rec, ext, cursor, pairs, cap, count, sc, order,
                  order_blocks);
    return 0;
}

}  // namespace soit
