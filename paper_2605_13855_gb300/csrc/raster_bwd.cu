// raster_bwd.cu -- backward of the OIT raster (App. B, Eq. 9-10; Sec. 4.2).
//
// Per-splat parallel: a tile's 256 pixel states are loaded into shared
// memory once; each warp takes 32 of the tile's splats (lane = splat) and
// walks the tile's rows, each lane evaluating its own splat at the pixels of
// the row.  Nothing is stored per pixel in the forward except the state, the
// per-pair alpha is recomputed from the same record, and each lane ends the
// tile with its splat's full tile gradient in registers, added with one
// vector atomic per 4 fields.  No pair is evaluated twice.
//
// Per pixel state (g = dL/dC), five values: B g (3), A = T g.(F - c0) and
// -B g.F, with B = (1 - T)/Q (0 if Q = 0).  Eq. 10 contracted with g gives,
// per pair, with D = B (g.c - g.F) = (B g).c + (-B g.F),
//   dL/da = A/(1 - a) + w D,  dL/dw = a D,  dL/dc = w a (B g),
// and, unless a is clamped at 0.99, dL/d(ln o) = a dL/da and
// dL/ds = -ln2 a dL/da, chained to (mu'x, mu'y, r, A2, B2) below.
//
// The warps take groups of 32 of the tile's splats and walk every pixel of
// the rows their lanes' ellipses reach (every lane evaluates the same pixels,
// so the state loads are broadcasts; a lane whose splat misses a pixel adds
// exact zeros there).  A vote per group of pixels, skipping the groups that no
// lane's ellipse reaches, saved under 1 % of the lane slots on the 1M-splat
// workload and cost more than that in votes, branches and live predicates.
// By default each chunk
// of up to 1024 of the tile's pairs is first counting-sorted in shared memory
// by where the splat starts in the tile (splats whose cutoff ellipse contains
// the whole tile first, then by first row), and the warps take consecutive
// groups from a shared counter, so that a warp's lanes reach similar rows;
// the launch option bwd_walk = 2 takes the pairs in arena order instead.
// Each lane evaluates two adjacent columns per step with paired FP32
// instructions (f32x2 FMA / multiply / add, one issue slot for two values);
// components of the paired operations round exactly like their scalar
// counterparts, so contribution decisions stay identical to the forward
// raster's.
#include "common.cuh"
#include "launch.h"
#include "pair_eval.cuh"

namespace soit {

// Per contributing pair, with a = min(ar, 0.99), ar = 2^(log2 o - s),
// s = e1^2 + e2^2, e1 = A2 u, e2 = B2 dy (u = dx - r dy):
//   da = dL/da * a (0 if clamped) = dL/d(ln o) of the pair, and
//   dL/ds = -ln2 da.  Summing K = -2 ln2 times
//     Se = sum da e1, Sey = sum da e1 dy, See = sum da e1^2,
//     Sdy = sum da dy, Sdyy = sum da dy^2
// (the dy sums taken per tile row, where dy is constant; per row See comes
// from sum da nlg - nlrow sum da, since the pixel's rounded exponent is
// nlg = e1^2 + nlrow, which saves the product da e1 per pixel) gives
//   dL/dmu'x = -K A2 Se,  dL/dmu'y = K (A2 r Se - B2^2 Sdy),
//   dL/dr = -K A2 Sey,    dL/dA2 = K See / A2,  dL/dB2 = K B2 Sdyy.

// Per-lane accumulators of one splat over the tile (see the sums above).
struct BwdAcc {
    float2 gw, gc0, gc1, gc2;
    float See, Se, Sey, Sd, Sdy, Sdyy;
};
struct BwdSplat {
    float2 A2p, wp, c0p, c1p, c2p;
    float A2dx0, dy0, rA2, B2, log2o;
};

// The state of two adjacent pixels (x, x + 1) of a row: B g (3 components), A
// and -B g.F, each as an f32x2 pair in column order.
struct PixPair {
    float2 b0, b1, b2, A, nbF;
};

// The tile's pixel state: five planes (B g0, B g1, B g2, A, -B g.F) of the
// 256 pixels, four adjacent pixels of a row per float4, so that five
// broadcast loads fetch the state of two steps.
struct TileState {
    float4 p[5][kTilePix / 4];
    // pixel pairs (2m, 2m + 1) and (2m + 2, 2m + 3) of row ky, m even
    __device__ __forceinline__ void get2(int ky, int m, PixPair &lo, PixPair &hi) const {
        const int kq = ky * (kTile / 4) + (m >> 1);
        const float4 u0 = p[0][kq], u1 = p[1][kq], u2 = p[2][kq], u3 = p[3][kq], u4 = p[4][kq];
        lo = {make_float2(u0.x, u0.y), make_float2(u1.x, u1.y), make_float2(u2.x, u2.y), make_float2(u3.x, u3.y),
              make_float2(u4.x, u4.y)};
        hi = {make_float2(u0.z, u0.w), make_float2(u1.z, u1.w), make_float2(u2.z, u2.w), make_float2(u3.z, u3.w),
              make_float2(u4.z, u4.w)};
    }
};

// The tile's pixel state from the view's five planes into shared memory (zero
// outside the view).
template <int kThreads>
__device__ __forceinline__ void load_tile_state(const ViewDesc &vd, int tx, int ty, TileState &S) {
#pragma unroll
    for (int t = threadIdx.x; t < kTilePix; t += kThreads) {
        const int x = tx * kTile + (t & (kTile - 1)), y = ty * kTile + (t >> 4);
        float st5[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
        if (x < vd.W && y < vd.H) {
            const int64_t HW = (int64_t)vd.W * vd.H, pix = (int64_t)y * vd.W + x;
            const float *st = vd.state;
#pragma unroll
            for (int k = 0; k < 5; ++k) st5[k] = st[k * HW + pix];
        }
#pragma unroll
        for (int k = 0; k < 5; ++k) reinterpret_cast<float *>(S.p[k])[t] = st5[k];
    }
}

// One step of a lane: pixels (2m, 2m + 1) of a row against the lane's splat,
// given their exponents and cutoff decisions; a pixel that does not
// contribute runs it with a = 0, which adds exact zeros.  kClamp: some lane's splat
// can reach the 0.99 clamp; without it min(a, 0.99) = a and the clamp
// selects are left out (same results).
template <bool kClamp>
__device__ __forceinline__ void bwd_step(const BwdSplat &bs, float2 e1, float2 nlg, bool in0, bool in1,
                                         const PixPair &ps, float2 &Rd, float2 &Re, float2 &Rn, BwdAcc &acc) {
    const float2 m1 = make_float2(-1.f, -1.f), one2 = make_float2(1.f, 1.f);
    const float ar0 = fast_exp2(-nlg.x), ar1 = fast_exp2(-nlg.y);
    float2 a, am;
    if (kClamp) {
        a = make_float2(in0 ? fminf(ar0, kAlphaMax) : 0.f, in1 ? fminf(ar1, kAlphaMax) : 0.f);
        // the alpha path (o, mu', conic) is off where alpha is clamped
        am = make_float2(ar0 > kAlphaMax ? 0.f : a.x, ar1 > kAlphaMax ? 0.f : a.y);
    } else {
        a = make_float2(in0 ? ar0 : 0.f, in1 ? ar1 : 0.f);
        am = a;
    }
    const float2 D = __ffma2_rn(ps.b0, bs.c0p, __ffma2_rn(ps.b1, bs.c1p, __ffma2_rn(ps.b2, bs.c2p, ps.nbF)));
    const float2 oma = __ffma2_rn(a, m1, one2);  // 1 - a
    const float2 inv = make_float2(fast_rcp(oma.x), fast_rcp(oma.y));
    const float2 dLda = __ffma2_rn(ps.A, inv, __fmul2_rn(bs.wp, D));
    acc.gw = __ffma2_rn(a, D, acc.gw);
    acc.gc0 = __ffma2_rn(a, ps.b0, acc.gc0);  // times w in the epilogue
    acc.gc1 = __ffma2_rn(a, ps.b1, acc.gc1);
    acc.gc2 = __ffma2_rn(a, ps.b2, acc.gc2);
    const float2 da = __fmul2_rn(dLda, am);
    Rd = __fadd2_rn(Rd, da);
    Re = __ffma2_rn(da, e1, Re);
    Rn = __ffma2_rn(da, nlg, Rn);  // e1^2 = nlg - nlrow: the row adds Rn - nlrow Rd to See
}

// Rows [rlo, rhi] of the tile.  kTest: test every pixel against the cutoff
// (the pair contributes iff its exponent reaches -log2 255); without it every
// pixel contributes (the warp's splats all contain the whole tile, or are
// empty records whose alpha is 0).  The eight steps of a row run without
// branches, so that their chains interleave.
template <bool kTest, bool kClamp>
__device__ __forceinline__ void bwd_rows(const BwdSplat &bs, const TileState &S, int rlo, int rhi, BwdAcc &acc) {
    const float2 zero2 = make_float2(0.f, 0.f);
    for (int ky = rlo; ky <= rhi; ++ky) {
        const RowTerms rt = row_terms(bs.A2dx0, bs.dy0, bs.rA2, bs.B2, bs.log2o, ky);
        const float2 e10p = make_float2(rt.e10, rt.e10), nlp = make_float2(rt.nlrow, rt.nlrow);
        float2 Rd = zero2, Re = zero2, Rn = zero2;
#pragma unroll
        for (int m0 = 0; m0 < kTile / 2; m0 += 4) {
            float2 e1[4], nlg[4];
            bool in[8];
#pragma unroll
            for (int h = 0; h < 4; ++h) {
                const float kx = (float)(2 * (m0 + h));
                e1[h] = __ffma2_rn(bs.A2p, make_float2(kx, kx + 1.f), e10p);
                nlg[h] = pair_nlg2(e1[h], nlp);
                in[2 * h] = !kTest || nlg[h].x <= kMaxNegLog2Alpha;
                in[2 * h + 1] = !kTest || nlg[h].y <= kMaxNegLog2Alpha;
            }
#pragma unroll
            for (int h = 0; h < 4; h += 2) {
                PixPair p0, p1;
                S.get2(ky, m0 + h, p0, p1);
                bwd_step<kClamp>(bs, e1[h], nlg[h], in[2 * h], in[2 * h + 1], p0, Rd, Re, Rn, acc);
                bwd_step<kClamp>(bs, e1[h + 1], nlg[h + 1], in[2 * h + 2], in[2 * h + 3], p1, Rd, Re, Rn, acc);
            }
        }
        const float rd = Rd.x + Rd.y, re = Re.x + Re.y, rn = Rn.x + Rn.y;
        acc.See += fmaf(-rt.nlrow, rd, rn);
        acc.Sd += rd;
        acc.Sdy = fmaf(rd, rt.dy, acc.Sdy);
        acc.Sdyy = fmaf(rd, rt.dy * rt.dy, acc.Sdyy);
        acc.Se += re;
        acc.Sey = fmaf(re, rt.dy, acc.Sey);
    }
}

// One warp's group of 32 splats (record indices q; >= nrec: no splat) over the tile.
__device__ __forceinline__ void bwd_group(const float4 *__restrict__ rec, uint32_t q, uint32_t nrec, float ox,
                                          float oy, const TileState &S, float4 *__restrict__ sgrad) {
    const bool valid = q < nrec;
    float4 a0 = make_float4(0.f, 0.f, 0.f, 1.f), a1 = make_float4(0.f, -INFINITY, 0.f, -1.f);
    float4 a2 = make_float4(0.f, 0.f, 0.f, 0.f);
    if (valid) {
        a0 = rec[3 * (int64_t)q + 0];
        a1 = rec[3 * (int64_t)q + 1];
        a2 = rec[3 * (int64_t)q + 2];
    }
    const float rr = a0.z, A2 = a0.w, B2 = a1.x, log2o = a1.y, w = a1.z, yh = a1.w;
    const SplatConsts sc = splat_consts(ox, oy, a0.x, a0.y, rr, A2);
    // rows of the tile this lane's ellipse can reach; the warp walks their union
    int rlo = kTile, rhi = -1;
    if (valid && yh >= 0.f) {
        rlo = f2i_clamped(ceilf(-yh - sc.dy0), 0, kTile);
        rhi = f2i_clamped(floorf(yh - sc.dy0), -1, kTile - 1);
    }
    rlo = __reduce_min_sync(0xffffffffu, rlo);
    rhi = __reduce_max_sync(0xffffffffu, rhi);
    if (rlo > rhi) return;  // uniform: no lane reaches the tile

    const float2 zero2 = make_float2(0.f, 0.f);
    BwdAcc acc;
    acc.gw = acc.gc0 = acc.gc1 = acc.gc2 = zero2;
    acc.See = acc.Se = acc.Sey = acc.Sd = acc.Sdy = acc.Sdyy = 0.f;
    const BwdSplat bs{make_float2(A2, A2), make_float2(w, w), make_float2(a2.x, a2.x), make_float2(a2.y, a2.y),
                      make_float2(a2.z, a2.z), sc.A2dx0, sc.dy0, sc.rA2, B2, log2o};
    // a splat with log2 o <= kNoClampLog2 never reaches the 0.99 clamp
    const bool clamp = __any_sync(0xffffffffu, valid && log2o > kNoClampLog2);
    const bool full = !valid || tile_inside(sc, A2, B2, log2o);
    if (__all_sync(0xffffffffu, full)) {  // every pixel of the tile contributes
        if (clamp)
            bwd_rows<false, true>(bs, S, 0, kTile - 1, acc);
        else
            bwd_rows<false, false>(bs, S, 0, kTile - 1, acc);
    } else if (clamp) {
        bwd_rows<true, true>(bs, S, rlo, rhi, acc);
    } else {
        bwd_rows<true, false>(bs, S, rlo, rhi, acc);
    }
    if (valid) {
        const float K = -2.f * kLn2;
        const float See1 = acc.See;
        const float g_mx = -K * A2 * acc.Se;
        const float g_my = K * (A2 * rr * acc.Se - B2 * B2 * acc.Sdy);
        const float g_r = -K * A2 * acc.Sey;
        const float g_A2 = K * See1 / A2;
        const float g_B2 = K * B2 * acc.Sdyy;
        float4 *out = sgrad + 3 * (int64_t)q;
        atomicAdd(out + 0, make_float4(g_mx, g_my, g_r, g_A2));
        atomicAdd(out + 1, make_float4(g_B2, acc.Sd, acc.gw.x + acc.gw.y, w * (acc.gc0.x + acc.gc0.y)));
        atomicAdd(reinterpret_cast<float2 *>(out + 2),
                  make_float2(w * (acc.gc1.x + acc.gc1.y), w * (acc.gc2.x + acc.gc2.y)));
    }
}

// Sort key of a pair (ascending): 0 when the splat's cutoff ellipse contains
// the whole tile, else 1 + the first tile row its ellipse reaches.
constexpr int kBwdKeys = kTile + 1;
__device__ __forceinline__ int pair_key(const float4 *rec, uint32_t q, float ox, float oy) {
    const float4 a0 = rec[3 * (int64_t)q + 0], a1 = rec[3 * (int64_t)q + 1];
    const float A2 = a0.w, B2 = a1.x, log2o = a1.y, yh = a1.w;
    const SplatConsts c = splat_consts(ox, oy, a0.x, a0.y, a0.z, A2);
    if (tile_inside(c, A2, B2, log2o)) return 0;
    return 1 + f2i_clamped(ceilf(-yh - c.dy0), 0, kTile - 1);
}

constexpr int kBwdChunk = 1024;  // pairs sorted together (the heaviest tile of 1M splats / 5 % holds ~900)
// Threads per block (one block per tile): four warps keep more of a typical tile's warps busy
// (the median tile holds ~110 splats at a 5 % active set) than eight, without stretching the
// heaviest tiles into long serial chains as two do.
constexpr int kBwdThreads = 128;
constexpr int kBwdMinBlocks = 7;  // <= 73 registers a thread (6 blocks: 1.5 % slower; 8: the same as 7)

// kSort: each chunk of up to kBwdChunk of the tile's pairs is counting-sorted in shared memory
// by pair_key before the warps take groups of 32 from a shared counter (else the warps take the
// pairs in arena order).
template <bool kSort>
__global__ void __launch_bounds__(kBwdThreads, kBwdMinBlocks)
    raster_bwd_kernel(const __grid_constant__ Batch b, const float4 *__restrict__ rec,
                      const int *__restrict__ offsets, const uint32_t *__restrict__ pairs, int64_t cap,
                      uint32_t nrec, float4 *__restrict__ sgrad, int *queue) {
    __shared__ TileState S;
    __shared__ uint32_t sorted[kSort ? kBwdChunk : 1];
    __shared__ uint16_t slot[kSort ? kBwdChunk : 1];
    __shared__ uint8_t keys[kSort ? kBwdChunk : 1];
    __shared__ int hist[32];
    __shared__ int next_group;

    __shared__ int item_s;
    if (bin_failed(b)) return;  // the binning scan gave up: offsets and tile order are incomplete
    // queue == null: this block's tile (block_tile); else a persistent block that takes tiles from the
    // queue (in the raster order) until none is left
    for (int it = 0;; ++it) {
        int gt;
        if (queue) {
            if (threadIdx.x == 0) item_s = atomicAdd(queue, 1);
            __syncthreads();  // also: every warp is done with the previous tile
            const int item = item_s;
            __syncthreads();
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
        const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
        // the pixel state is the forward raster's output: it is loaded after pdl_wait, once the
        // tile's pairs are sorted (pairs, records and tile order are older, the scatter's and the
        // projection's), so that the sort overlaps the end of the forward
        bool have_state = false;
        auto state_in = [&]() {
            if (have_state) return;
            pdl_wait();
            pdl_allow_next();
            load_tile_state<kBwdThreads>(vd, tx, ty, S);
            have_state = true;
        };

        const int start = offsets[gt];
        const int end = (int)min((int64_t)offsets[gt + 1], cap);
        const float ox = (float)(tx * kTile) + 0.5f, oy = (float)(ty * kTile) + 0.5f;

        if constexpr (!kSort) {
            if (start < end) state_in();
            __syncthreads();
            for (int cb0 = start + warp * 32; cb0 < end; cb0 += kBwdThreads) {
                const int idx = cb0 + lane;
                bwd_group(rec, idx < end ? pairs[idx] : 0xffffffffu, nrec, ox, oy, S, sgrad);
            }
        } else {
            for (int c0 = start; c0 < end; c0 += kBwdChunk) {
                const int nc = min(kBwdChunk, end - c0);
                if (c0 > start) __syncthreads();  // the previous chunk's arrays are consumed
                if (tid < 32) hist[tid] = 0;
                if (tid == 0) next_group = 0;
                __syncthreads();
                for (int i = tid; i < nc; i += kBwdThreads) {
                    const uint32_t q = pairs[c0 + i];
                    const int key = q < nrec ? pair_key(rec, q, ox, oy) : kBwdKeys - 1;
                    keys[i] = (uint8_t)key;
                    slot[i] = (uint16_t)atomicAdd(&hist[key], 1);
                }
                __syncthreads();
                if (warp == 0) {  // first position of each key
                    const int h = hist[lane];
                    int incl = h;
    #pragma unroll
                    for (int off = 1; off < 32; off <<= 1) {
                        const int y = __shfl_up_sync(0xffffffffu, incl, off);
                        if (lane >= off) incl += y;
                    }
                    hist[lane] = incl - h;
                }
                __syncthreads();
                for (int i = tid; i < nc; i += kBwdThreads) sorted[hist[keys[i]] + slot[i]] = pairs[c0 + i];
                state_in();
                __syncthreads();  // the sorted pairs and the state
                for (;;) {
                    int g = 0;
                    if (lane == 0) g = atomicAdd(&next_group, 1);
                    g = __shfl_sync(0xffffffffu, g, 0);
                    const int idx = g * 32 + lane;
                    if (g * 32 >= nc) break;  // uniform over the warp
                    bwd_group(rec, idx < nc ? sorted[idx] : 0xffffffffu, nrec, ox, oy, S, sgrad);
                }
            }
        }
    }
}

// Unfused backward: turn the forward's (F, T, Q) planes and dL/dC into the
// pixel state, in place.
__global__ void prep_state_kernel(const __grid_constant__ Batch b, float bg0, float bg1, float bg2) {
    const int v = blockIdx.y;
    if (v >= b.n_views) return;
    const ViewDesc &vd = b.v[v];
    const int64_t HW = (int64_t)vd.W * vd.H;
    for (int64_t pix = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; pix < HW;
         pix += (int64_t)gridDim.x * blockDim.x) {
        float *st = vd.state;
        const float F0 = st[pix], F1 = st[HW + pix], F2 = st[2 * HW + pix], T = st[3 * HW + pix], Q = st[4 * HW + pix];
        const float *gi = vd.grad_image + 3 * pix;
        const float g0 = gi[0], g1 = gi[1], g2 = gi[2];
        const float B = Q > 0.f ? (1.f - T) / Q : 0.f;
        st[pix] = B * g0;
        st[HW + pix] = B * g1;
        st[2 * HW + pix] = B * g2;
        st[3 * HW + pix] = T * (g0 * (F0 - bg0) + g1 * (F1 - bg1) + g2 * (F2 - bg2));
        st[4 * HW + pix] = -B * (g0 * F0 + g1 * F1 + g2 * F2);
    }
}

int launch_prep_state(const Batch &b, const float bg[3], cudaStream_t st) {
    prep_state_kernel<<<dim3(304, b.n_views), 256, 0, st>>>(b, bg[0], bg[1], bg[2]);
    return 0;
}

template <bool kSort>
static void launch_bwd(const Batch &b, const float4 *rec, const int *offsets, const uint32_t *pairs, int64_t cap,
                       uint32_t nrec, float4 *sgrad, int *queue, bool pdl, cudaStream_t st) {
    auto kern = raster_bwd_kernel<kSort>;
    int grid = b.total_tiles;
    if (queue) {  // persistent: as many blocks as fit on the device at once, at most one per tile
        int dev = 0, sms = 0, per_sm = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kBwdThreads, 0);
        const int g = (per_sm > 0 ? per_sm : 1) * (sms > 0 ? sms : 1);
        grid = g < grid ? g : grid;
        cudaMemsetAsync(queue, 0, sizeof(int), st);
        pdl = false;  // the operation just before the raster is this memset
    }
    launch_kernel(kern, dim3(grid), dim3(kBwdThreads), st, pdl, b, rec, offsets, pairs, cap, nrec, sgrad, queue);
}

int launch_raster_bwd(const Batch &b, int walk, const float4 *rec, const int *offsets, const uint32_t *pairs,
                      int64_t cap, float4 *sgrad, int *queue, bool pdl, cudaStream_t st) {
    if (b.total_tiles == 0) return 0;
    const uint32_t nrec = (uint32_t)((int64_t)b.n_views * b.n_list);
    if (walk == kBwdWalkArena)
        launch_bwd<false>(b, rec, offsets, pairs, cap, nrec, sgrad, queue, pdl, st);
    else
        launch_bwd<true>(b, rec, offsets, pairs, cap, nrec, sgrad, queue, pdl, st);
    return 0;
}

}  // namespace soit
