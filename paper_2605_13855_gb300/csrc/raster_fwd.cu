// raster_fwd.cu -- tile rasteriser of the OIT sums (Alg. 2 BAN / BAU, Eq. 7).
//
// One block per 16x16 tile; each thread owns a 1xS strip of pixels of one
// row (S = 1, 2 or 4, a launch parameter; the exponent of each pixel of the
// strip costs two FMAs), each warp owns 2S rows.  The tile's records are
// staged through shared memory 128 at a time, already shifted to
// tile-relative offsets, and sorted by warp ballots into one list of the
// records whose cutoff ellipse contains the whole tile (evaluated without
// cutoff tests) and, per warp, a list of the other records that reach its
// rows; each warp walks its lists four records per branch-free iteration.  Every
// pixel accumulates over the tile's splats P += a w c, Q += a w and
// T *= (1 - a) (log T += log(1 - a) for the frozen sums), the sums taken in
// 32-splat blocks added to the total, so that the FP32 rounding of sums over
// thousands of splats stays at the level of about 32 + n/32 additions.  The epilogue depends on the mode:
//   kRasterFused: combine with the view's frozen sums (P_F, Q_F, log T_F),
//     write C = T c0 + (1 - T) P/Q, the L1 loss and the backward pixel state
//     (g, A = T g.(F - c0), B = (1 - T)/Q, g.F) with g = sign(C - I)/(3HW).
//   kRasterAux: as fused but without a target; writes (F, T, Q) for the
//     backward to turn into the state once dL/dC is known.
//   kRasterSums: the records carry a sign s = +-1; adds s a w c, s a w and
//     s log(1 - a) to the frozen planes (the delayed pre-render update).
#include "common.cuh"
#include "launch.h"
#include "pair_eval.cuh"

namespace soit {

// Records staged per round.  128 keeps a block's shared memory at 12 KB, so that with the strip
// of 4 pixels 12 blocks (24 warps, 80 registers a thread) fit an SM; 256 records at 19 KB allowed
// 9 (106 registers) and measured 5 % slower on the 1M-splat / 5 % workload.
constexpr int kFwdBatch = 128;
constexpr int kFwdUnroll = 4;     // records per iteration of the accumulation loop

// The strip's negated exponents nlg = -log2 alpha_raw = e1^2 + nlrow, two
// pixels per f32x2 instruction where the strip has pairs (each component
// rounds like the scalar FMA, so the decisions match the backward's).
template <int kStrip>
__device__ __forceinline__ void strip_exponents(float A2, float e10, float nlrow, int sx, float *nlg) {
    if (kStrip == 1) {
        nlg[0] = pair_nlg(col_e1(A2, e10, sx), nlrow);
    } else {
        const float2 A2p = make_float2(A2, A2), e10p = make_float2(e10, e10), nlp = make_float2(nlrow, nlrow);
#pragma unroll
        for (int p = 0; p < kStrip; p += 2) {
            const float2 e1 = __ffma2_rn(A2p, make_float2((float)(sx + p), (float)(sx + p + 1)), e10p);
            const float2 l = pair_nlg2(e1, nlp);
            nlg[p] = l.x;
            nlg[p + 1] = l.y;
        }
    }
}

// One staged record j against the thread's strip, accumulated into the
// 32-splat block partials.  kTest: test every pixel against the cutoff
// (without it the record's ellipse contains the whole tile).  The body has no
// branches, so that the compiler can interleave two records.
template <int kMode, bool kCount, int kStrip, bool kTest, bool kClamp>
__device__ __forceinline__ void fwd_splat(const float4 *s0, const float4 *s1, const float4 *s2, const float *ssign,
                                          int j, int ky, int sx, bool in_view_row, int x0, int W, float2 *b01,
                                          float2 *b2q, float *bl, float *T, unsigned &n_contrib) {
    const float4 a0 = s0[j], a1 = s1[j], a2 = s2[j];
    const bool counted = kCount && j < kFwdBatch && in_view_row;  // the empty record counts nothing
    const RowTerms rt = row_terms(a0.x, a0.y, a0.z, a1.x, a1.z, ky);
    float nlg[kStrip];
    strip_exponents<kStrip>(a0.w, rt.e10, rt.nlrow, sx, nlg);
#pragma unroll
    for (int p = 0; p < kStrip; ++p) {
        if (!kTest || nlg[p] <= kMaxNegLog2Alpha) {
            const float ar = fast_exp2(-nlg[p]);
            const float a = kClamp ? fminf(ar, kAlphaMax) : ar;
            const float2 aa = make_float2(a, a);
            b01[p] = __ffma2_rn(aa, make_float2(a2.x, a2.y), b01[p]);
            b2q[p] = __ffma2_rn(aa, make_float2(a2.z, a2.w), b2q[p]);
            if (kMode == kRasterSums)
                bl[p] = fmaf(ssign[j], log1pf(-a), bl[p]);
            else
                T[p] = fmaf(-T[p], a, T[p]);
            if (kCount) n_contrib += (counted && x0 + p < W) ? 1u : 0u;
        }
    }
}

// A list of staged records (indices into the staged arrays) into the
// thread's strip, kFwdUnroll records per iteration (the list is padded to a
// multiple of kFwdUnroll with the empty record at index kFwdBatch), summed in
// 32-record blocks that are added to the totals (two-level summation).
template <int kMode, bool kCount, int kStrip, bool kTest, bool kClamp>
__device__ __forceinline__ void fwd_list(const float4 *s0, const float4 *s1, const float4 *s2, const float *ssign,
                                         const uint16_t *list, int cnt, int ky, int sx, bool in_view_row, int x0,
                                         int W, float2 *P01, float2 *P2Q, float *T, unsigned &n_contrib) {
    for (int jb = 0; jb < cnt; jb += 32) {
        float2 b01[kStrip], b2q[kStrip];
        float bl[kStrip];
#pragma unroll
        for (int p = 0; p < kStrip; ++p) {
            b01[p] = b2q[p] = make_float2(0.f, 0.f);
            bl[p] = 0.f;
        }
        const int je = min(cnt, jb + 32);
        for (int i = jb; i < je; i += kFwdUnroll) {
#pragma unroll
            for (int u = 0; u < kFwdUnroll; ++u) {
                const int j = list[i + u];
                fwd_splat<kMode, kCount, kStrip, kTest, kClamp>(s0, s1, s2, ssign, j, ky, sx, in_view_row, x0, W,
                                                                b01, b2q, bl, T, n_contrib);
            }
        }
#pragma unroll
        for (int p = 0; p < kStrip; ++p) {
            P01[p] = __fadd2_rn(P01[p], b01[p]);
            P2Q[p] = __fadd2_rn(P2Q[p], b2q[p]);
            if (kMode == kRasterSums) T[p] += bl[p];
        }
    }
}

// Append the staging lanes whose flag is set to a shared list (warp ballot,
// one shared atomic per warp).
__device__ __forceinline__ void list_append(bool flag, int k, int *cnt, uint16_t *list) {
    const int lane = threadIdx.x & 31;
    const unsigned bal = __ballot_sync(0xffffffffu, flag);
    int wb = 0;
    if (lane == 0 && bal) wb = atomicAdd(cnt, __popc(bal));
    wb = __shfl_sync(0xffffffffu, wb, 0);
    if (flag) list[wb + __popc(bal & ((1u << lane) - 1u))] = (uint16_t)k;
}

// Blocks per SM asked of the compiler: 12 for the 4-pixel strip (at most 80 registers; 14 blocks
// at 72 registers and 16 at 64 spill and measured slower).
template <int kMode, bool kCount, int kStrip>
__global__ void __launch_bounds__(kTilePix / kStrip, kStrip == 1 ? 4 : (kStrip == 2 ? 4 : 12)) raster_fwd_kernel(const __grid_constant__ Batch b,
                                                                 const float4 *__restrict__ rec,
                                                                 const int *__restrict__ offsets,
                                                                 const uint32_t *__restrict__ pairs, int64_t cap,
                                                                 uint32_t nrec, float bg0, float bg1, float bg2,
                                                                 float *loss, unsigned long long *contrib,
                                                                 int *queue) {
    constexpr int kFwdThreads = kTilePix / kStrip;
    constexpr int kStripsPerRow = kTile / kStrip;
    constexpr int kWarps = kFwdThreads / 32;
    constexpr int kRowsPerWarp = kTile / kWarps;
    // staged records; index kFwdBatch is an empty record (alpha 0 at every pixel)
    __shared__ float4 s0[kFwdBatch + 1], s1[kFwdBatch + 1], s2[kFwdBatch + 1];
    __shared__ float ssign[kMode == kRasterSums ? kFwdBatch + 1 : 1];
    // per batch: the records whose cutoff ellipse contains the whole tile (every warp takes them
    // without cutoff tests), and per warp the other records whose ellipse reaches its rows
    __shared__ uint16_t flist[kFwdBatch + kFwdUnroll], wlist[kWarps][kFwdBatch + kFwdUnroll];
    __shared__ int fcnt, wcnt[kWarps];
    __shared__ float red[kFwdThreads / 32];
    // the tile's sums (P_r, P_g, P_b, Q, T or log T) by pixel, for the epilogue's row-contiguous mapping
    __shared__ float psum[5][kTilePix];
    __shared__ unsigned red_n[kFwdThreads / 32];

    __shared__ int item_s;
    pdl_wait();  // the scatter's pairs and tile order
    pdl_allow_next();
    if (bin_failed(b)) return;  // the binning scan gave up: offsets and tile order are incomplete
    // queue == null: this block's tile (block_tile); else a persistent block that takes tiles from the
    // queue (in the raster order) until none is left
    for (int it = 0;; ++it) {
        int gt;
        if (queue) {
            if (threadIdx.x == 0) item_s = atomicAdd(queue, 1);
            __syncthreads();
            const int item = item_s;
            __syncthreads();  // item_s is read before it is taken again
            if (item >= b.total_tiles) break;
            gt = b.tile_order ? __ldg(b.tile_order + item) : item;
        } else {
            if (it > 0) break;
            gt = block_tile(b);
        }
        const int v = find_view(b, gt);
        const ViewDesc &vd = b.v[v];
        const int lt = gt - vd.tile_base;
        const int ty = lt / vd.tiles_x, tx = lt - ty * vd.tiles_x;
        const int tid = threadIdx.x, warp = tid >> 5;
        const int ky = tid / kStripsPerRow, sx = (tid % kStripsPerRow) * kStrip;
        const float ox = (float)(tx * kTile) + 0.5f, oy = (float)(ty * kTile) + 0.5f;
        const bool in_view_row = ty * kTile + ky < vd.H;
        const int x0 = tx * kTile + sx;

        const int start = offsets[gt];
        const int end = (int)min((int64_t)offsets[gt + 1], cap);

        if (tid == 0) {
            s0[kFwdBatch] = make_float4(0.f, 0.f, 0.f, 0.f);
            s1[kFwdBatch] = make_float4(0.f, 0.f, -INFINITY, -1.f);  // log2 o = -inf: alpha 0
            s2[kFwdBatch] = make_float4(0.f, 0.f, 0.f, 0.f);
            if (kMode == kRasterSums) ssign[kFwdBatch] = 0.f;
        }

        // per pixel: (P_r, P_g) and (P_b, Q) as f32x2 pairs (one paired FMA per pair of sums;
        // each component rounds like the scalar FMA), T (log T in sums mode)
        float2 P01[kStrip], P2Q[kStrip];
        float T[kStrip];
    #pragma unroll
        for (int j = 0; j < kStrip; ++j) {
            P01[j] = P2Q[j] = make_float2(0.f, 0.f);
            T[j] = kMode == kRasterSums ? 0.f : 1.f;  // log T in sums mode
        }
        unsigned n_contrib = 0;

        for (int base = start; base < end; base += kFwdBatch) {
            const int n = min(kFwdBatch, end - base);
            __syncthreads();  // the previous batch's records and lists are consumed
            if (tid == 0) fcnt = 0;
            if (tid < kWarps) wcnt[tid] = 0;
            __syncthreads();
            int may_clamp = 0;  // some staged splat can reach the 0.99 clamp
            for (int k0 = 0; k0 < n; k0 += 2 * kFwdThreads) {  // uniform trip count: the lists use warp ballots
                // two records a thread: both pair indices, then both records, are loaded before use
                uint32_t qv[2];
                float4 r0[2], r1[2], r2[2];
#pragma unroll
                for (int u = 0; u < 2; ++u) {
                    const int k = k0 + u * kFwdThreads + tid;
                    qv[u] = k < n ? pairs[base + k] : 0xffffffffu;
                }
#pragma unroll
                for (int u = 0; u < 2; ++u) {
                    r0[u] = make_float4(0.f, 0.f, 0.f, 0.f);
                    r1[u] = r2[u] = r0[u];
                    if (qv[u] < nrec) {
                        r0[u] = rec[3 * (int64_t)qv[u] + 0];
                        r1[u] = rec[3 * (int64_t)qv[u] + 1];
                        r2[u] = rec[3 * (int64_t)qv[u] + 2];
                    }
                }
#pragma unroll
                for (int u = 0; u < 2; ++u) {
                    const int k = k0 + u * kFwdThreads + tid;
                    // staged: s0 = (A2 dx0, dy0, r A2, A2), s1 = (B2, 0, log2 o, yh),
                    //         s2 = (w c_r, w c_g, w c_b, w) (times the sign in sums mode)
                    bool ok = false, full = false;
                    float dy0 = 0.f, yh = -1.f;
                    if (k < n) {
                        const uint32_t q = qv[u];
                        float4 t0 = make_float4(0.f, 0.f, 0.f, 0.f), t1 = make_float4(0.f, 0.f, -INFINITY, -1.f);
                        float4 t2 = make_float4(0.f, 0.f, 0.f, 0.f);
                        if (q < nrec) {  // never written by this call's scatter otherwise: contributes nothing
                            const float4 a0 = r0[u];
                            const float4 a1 = r1[u];
                            const float4 a2 = r2[u];
                            const SplatConsts c = splat_consts(ox, oy, a0.x, a0.y, a0.z, a0.w);
                            t0 = make_float4(c.A2dx0, c.dy0, c.rA2, a0.w);
                            t1 = make_float4(a1.x, 0.f, a1.y, a1.w);
                            ok = true;
                            // the whole tile inside the cutoff ellipse (its four corner pixels are, by a margin)
                            full = tile_inside(c, a0.w, a1.x, a1.y);
                            dy0 = c.dy0;
                            yh = a1.w;
                            may_clamp |= a1.y > kNoClampLog2 ? 1 : 0;
                            const float ws = kMode == kRasterSums ? a1.z * a2.w : a1.z;
                            t2 = make_float4(ws * a2.x, ws * a2.y, ws * a2.z, ws);
                            if (kMode == kRasterSums) ssign[k] = a2.w;
                        }
                        s0[k] = t0;
                        s1[k] = t1;
                        s2[k] = t2;
                    }
                    list_append(ok && full, k, &fcnt, flist);
#pragma unroll
                    for (int w = 0; w < kWarps; ++w) {
                        // the ellipse's rows |dy0 + ky| <= yh reach rows [w R, w R + R - 1] of the tile
                        const float dlo = dy0 + (float)(w * kRowsPerWarp);
                        const bool hit = ok && !full && !(dlo > yh || dlo + (float)(kRowsPerWarp - 1) < -yh);
                        list_append(hit, k, &wcnt[w], wlist[w]);
                    }
                }
            }
            const bool clamp = __syncthreads_or(may_clamp) != 0;
            const int nf0 = fcnt, nw0 = wcnt[warp];
            // pad both lists of this warp to a multiple of kFwdUnroll with the empty record (every
            // warp pads the shared list with the same values past its end)
            if ((tid & 31) < kFwdUnroll - 1) {
                flist[nf0 + (tid & 31)] = (uint16_t)kFwdBatch;
                wlist[warp][nw0 + (tid & 31)] = (uint16_t)kFwdBatch;
            }
            __syncwarp();
            const int nf = (nf0 + kFwdUnroll - 1) & ~(kFwdUnroll - 1), nw = (nw0 + kFwdUnroll - 1) & ~(kFwdUnroll - 1);
            if (clamp) {
                fwd_list<kMode, kCount, kStrip, false, true>(s0, s1, s2, ssign, flist, nf, ky, sx, in_view_row, x0, vd.W,
                                                             P01, P2Q, T, n_contrib);
                fwd_list<kMode, kCount, kStrip, true, true>(s0, s1, s2, ssign, wlist[warp], nw, ky, sx, in_view_row, x0,
                                                            vd.W, P01, P2Q, T, n_contrib);
            } else {
                fwd_list<kMode, kCount, kStrip, false, false>(s0, s1, s2, ssign, flist, nf, ky, sx, in_view_row, x0,
                                                              vd.W, P01, P2Q, T, n_contrib);
                fwd_list<kMode, kCount, kStrip, true, false>(s0, s1, s2, ssign, wlist[warp], nw, ky, sx, in_view_row, x0,
                                                             vd.W, P01, P2Q, T, n_contrib);
            }
        }

        // the sums to shared memory, then the epilogue with a thread per pixel and consecutive
        // threads on consecutive pixels of a row: each load and store of a plane covers two
        // contiguous row segments per warp (a thread's own strip would scatter them over 8 rows)
#pragma unroll
        for (int p = 0; p < kStrip; ++p) {
            const int i = ky * kTile + sx + p;
            psum[0][i] = P01[p].x;
            psum[1][i] = P01[p].y;
            psum[2][i] = P2Q[p].x;
            psum[3][i] = P2Q[p].y;
            psum[4][i] = T[p];
        }
        __syncthreads();
        const int64_t HW = (int64_t)vd.W * vd.H;
        float my_loss = 0.f;
        const float inv3hw = 1.f / (3.f * (float)HW);
    #pragma unroll
        for (int i = tid; i < kTilePix; i += kFwdThreads) {
            const int x = tx * kTile + (i & (kTile - 1)), y = ty * kTile + i / kTile;
            if (x >= vd.W || y >= vd.H) continue;
            const int64_t pix = (int64_t)y * vd.W + x;
            const float p0 = psum[0][i], p1 = psum[1][i], p2 = psum[2][i], pq = psum[3][i], pt = psum[4][i];
            if (kMode == kRasterSums) {
                float *fz = vd.frozen;
                fz[pix] += p0;
                fz[HW + pix] += p1;
                fz[2 * HW + pix] += p2;
                fz[3 * HW + pix] += pq;
                fz[4 * HW + pix] += pt;
            } else {
                // the frozen complement's sums (none when the whole set is rendered)
                const float *fz = vd.frozen;
                const float f0 = fz ? fz[pix] : 0.f, f1 = fz ? fz[HW + pix] : 0.f, f2 = fz ? fz[2 * HW + pix] : 0.f;
                const float fq = fz ? fz[3 * HW + pix] : 0.f;
                const float Pt0 = p0 + f0, Pt1 = p1 + f1, Pt2 = p2 + f2;
                const float Qt = pq + fq;
                const float Tt = fz ? pt * expf(fz[4 * HW + pix]) : pt;
                const float invQ = Qt > 0.f ? 1.f / Qt : 0.f;
                const float F0 = Pt0 * invQ, F1 = Pt1 * invQ, F2 = Pt2 * invQ;
                const float omT = 1.f - Tt;
                const float C0 = fmaf(Tt, bg0, omT * F0), C1 = fmaf(Tt, bg1, omT * F1), C2 = fmaf(Tt, bg2, omT * F2);
                float *img = vd.image + 3 * pix;
                img[0] = C0;
                img[1] = C1;
                img[2] = C2;
                float *st = vd.state;
                if (kMode == kRasterFused) {
                    const float *tg = vd.target + 3 * pix;
                    const float d0 = C0 - tg[0], d1 = C1 - tg[1], d2 = C2 - tg[2];
                    my_loss += fabsf(d0) + fabsf(d1) + fabsf(d2);
                    const float g0 = d0 > 0.f ? inv3hw : (d0 < 0.f ? -inv3hw : 0.f);
                    const float g1 = d1 > 0.f ? inv3hw : (d1 < 0.f ? -inv3hw : 0.f);
                    const float g2 = d2 > 0.f ? inv3hw : (d2 < 0.f ? -inv3hw : 0.f);
                    const float B = omT * invQ;
                    st[pix] = B * g0;
                    st[HW + pix] = B * g1;
                    st[2 * HW + pix] = B * g2;
                    st[3 * HW + pix] = Tt * (g0 * (F0 - bg0) + g1 * (F1 - bg1) + g2 * (F2 - bg2));
                    st[4 * HW + pix] = -B * (g0 * F0 + g1 * F1 + g2 * F2);
                } else {
                    st[pix] = F0;
                    st[HW + pix] = F1;
                    st[2 * HW + pix] = F2;
                    st[3 * HW + pix] = Tt;
                    st[4 * HW + pix] = Qt;
                }
            }
        }
        if ((kMode == kRasterFused && loss) || kCount) {
            float l = my_loss;
            unsigned c = n_contrib;
    #pragma unroll
            for (int off = 16; off > 0; off >>= 1) {
                l += __shfl_xor_sync(0xffffffffu, l, off);
                c += __shfl_xor_sync(0xffffffffu, c, off);
            }
            if ((tid & 31) == 0) {
                red[tid >> 5] = l;
                red_n[tid >> 5] = c;
            }
            __syncthreads();
            if (tid == 0) {
                float ls = 0.f;
                unsigned long long cs = 0;
                for (int k = 0; k < kFwdThreads / 32; ++k) {
                    ls += red[k];
                    cs += red_n[k];
                }
                if (kMode == kRasterFused && loss && ls != 0.f) atomicAdd(loss, ls * inv3hw);
                if (kCount && contrib && cs) atomicAdd(contrib, cs);
            }
        }
    }
}

// Persistent launch: as many blocks as fit on the device at once (occupancy x SMs), at most one per tile.
template <typename K>
static int persistent_grid(K kernel, int threads, int total_tiles) {
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, 0);
    const int g = (per_sm > 0 ? per_sm : 1) * (sms > 0 ? sms : 1);
    return g < total_tiles ? g : total_tiles;
}

template <int kMode, bool kCount, int kStrip>
static void launch_one(const Batch &b, const float4 *rec, const int *offsets, const uint32_t *pairs, int64_t cap,
                       uint32_t nrec, const float bg[3], float *loss, unsigned long long *contrib, int *queue,
                       bool pdl, cudaStream_t st) {
    constexpr int kThreads = kTilePix / kStrip;
    auto kern = raster_fwd_kernel<kMode, kCount, kStrip>;
    const int grid = queue ? persistent_grid(kern, kThreads, b.total_tiles) : b.total_tiles;
    launch_kernel(kern, dim3(grid), dim3(kThreads), st, pdl, b, rec, offsets, pairs, cap, nrec, bg[0], bg[1], bg[2],
                  loss, contrib, queue);
}

template <int kMode, int kStrip>
static void launch_strip(const Batch &b, bool count, const float4 *rec, const int *offsets, const uint32_t *pairs,
                         int64_t cap, uint32_t nrec, const float bg[3], float *loss, unsigned long long *contrib,
                         int *queue, bool pdl, cudaStream_t st) {
    if (count)
        launch_one<kMode, true, kStrip>(b, rec, offsets, pairs, cap, nrec, bg, loss, contrib, queue, pdl, st);
    else
        launch_one<kMode, false, kStrip>(b, rec, offsets, pairs, cap, nrec, bg, loss, contrib, queue, pdl, st);
}

template <int kMode>
static void launch_mode(const Batch &b, int strip, bool count, const float4 *rec, const int *offsets,
                        const uint32_t *pairs, int64_t cap, uint32_t nrec, const float bg[3], float *loss,
                        unsigned long long *contrib, int *queue, bool pdl, cudaStream_t st) {
    if (strip == 4)
        launch_strip<kMode, 4>(b, count, rec, offsets, pairs, cap, nrec, bg, loss, contrib, queue, pdl, st);
    else if (strip == 2)
        launch_strip<kMode, 2>(b, count, rec, offsets, pairs, cap, nrec, bg, loss, contrib, queue, pdl, st);
    else
        launch_strip<kMode, 1>(b, count, rec, offsets, pairs, cap, nrec, bg, loss, contrib, queue, pdl, st);
}

int launch_raster_fwd(const Batch &b, int mode, int strip, const float4 *rec, const int *offsets,
                      const uint32_t *pairs, int64_t cap, const float bg[3], float *loss, unsigned long long *contrib,
                      int *queue, bool pdl, cudaStream_t st) {
    if (b.total_tiles == 0) return 0;
    const uint32_t nrec = (uint32_t)((int64_t)b.n_views * b.n_list);
    const bool count = contrib != nullptr;
    if (queue) {
        cudaMemsetAsync(queue, 0, sizeof(int), st);
        pdl = false;  // the operation just before the raster is this memset, not the scatter
    }
    switch (mode) {
        case kRasterFused:
            launch_mode<kRasterFused>(b, strip, count, rec, offsets, pairs, cap, nrec, bg, loss, contrib, queue, pdl,
                                      st);
            break;
        case kRasterAux:
            launch_mode<kRasterAux>(b, strip, count, rec, offsets, pairs, cap, nrec, bg, loss, contrib, queue, pdl,
                                    st);
            break;
        default:
            launch_mode<kRasterSums>(b, strip, false, rec, offsets, pairs, cap, nrec, bg, nullptr, nullptr, queue,
                                     pdl, st);
            break;
    }
    return 0;
}

}  // namespace soit
