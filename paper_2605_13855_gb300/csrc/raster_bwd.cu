// raster_bwd.cu -- backward of the OIT raster (App. B, Eq. 9-10; Sec. 4.2).
//
// Per-splat parallel: a tile's 256 pixel states are loaded into shared
// memory once; each warp takes 32 of the tile's splats (lane = splat) and
// walks the tile's pixels, reading each pixel's state as a shared-memory
// broadcast.  Nothing is stored per pixel in the forward except the state,
// the per-pair alpha is recomputed from the same record, and each lane ends
// the tile with its splat's full tile gradient in registers, added with one
// vector atomic per 4 fields.  No pair is evaluated twice.
//
// Per pixel state (g = dL/dC), five planes: B g (3), A = T g.(F - c0) and
// -B g.F, with B = (1 - T)/Q (0 if Q = 0).  Eq. 10 contracted with g gives,
// per pair, with D = B (g.c - g.F) = (B g).c + (-B g.F),
//   dL/da = A/(1 - a) + w D,  dL/dw = a D,  dL/dc = w a (B g),
// and, unless a is clamped at 0.99, dL/d(ln o) = a dL/da and
// dL/ds = -ln2 a dL/da, chained to (mu'x, mu'y, r, A2, B2) below.  Each warp
// walks only the tile rows that some lane's ellipse reaches.
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
// (the dy sums taken per tile row, where dy is constant) gives
//   dL/dmu'x = -K A2 Se,  dL/dmu'y = K (A2 r Se - B2^2 Sdy),
//   dL/dr = -K A2 Sey,    dL/dA2 = K See / A2,  dL/dB2 = K B2 Sdyy.
// kGroup: before a round of the tile's splats (one per thread) is split into warps, a
// shared-memory counting sort puts first the splats whose cutoff ellipse
// contains the whole tile, then the others by the 4x4-pixel cell of the tile
// that holds their centre (clamped).  A warp whose splats all contain the
// tile evaluates every pixel without the cutoff test (no divergence); the
// others tend to share rows and columns.
//
// Each lane evaluates two adjacent columns per step with paired FP32
// instructions (f32x2 FMA / multiply / add, one issue slot for two values);
// the pixel states sit in shared memory as planes, so that one 128-bit
// broadcast load fetches a component for two steps.
// Components of the paired operations round exactly like their scalar
// counterparts, so contribution decisions stay identical to the forward
// raster's.
constexpr int kBwdKeys = 18;  // splat classes of the optional per-round ordering

// Per-lane accumulators of one splat over the tile (see the sums above).
struct BwdAcc {
    float2 See, gw, gc0, gc1, gc2;
    float Se, Sey, Sd, Sdy, Sdyy;
};
struct BwdSplat {
    float2 A2p, wp, l2op, c0p, c1p, c2p;
    float A2dx0, dy0, rA2, B2, thr;
};

// Pixel state of the tile: five planes (B g0, B g1, B g2, A, -B g.F), four
// adjacent pixels of a row per float4, so that five broadcast loads fetch
// the state of two steps.
struct BwdState {
    float4 p[5][kTilePix / 4];
};

// One step of a lane: pixels (2k, 2k + 1) of a row against the lane's splat,
// given their exponents and cutoff decisions; lanes without a contributing
// pixel run it with a = 0, which adds exact zeros.  kClamp: some lane's splat
// can reach the 0.99 clamp; without it min(a, 0.99) = a and the clamp
// selects are left out (same results).
template <bool kClamp>
__device__ __forceinline__ void bwd_step(const BwdSplat &bs, float2 e1, float2 sq, bool in0, bool in1, float2 b0,
                                         float2 b1, float2 b2, float2 Ap, float2 nbF, float2 &Rd, float2 &Re,
                                         BwdAcc &acc) {
    const float2 m1 = make_float2(-1.f, -1.f), one2 = make_float2(1.f, 1.f);
    // log2 o - s: -s + log2 o rounds once, exactly like the forward's subtraction
    const float2 lg = __ffma2_rn(sq, m1, bs.l2op);
    const float ar0 = fast_exp2(lg.x), ar1 = fast_exp2(lg.y);
    float2 a, am;
    if (kClamp) {
        a = make_float2(in0 ? fminf(ar0, kAlphaMax) : 0.f, in1 ? fminf(ar1, kAlphaMax) : 0.f);
        // the alpha path (o, mu', conic) is off where alpha is clamped
        am = make_float2(ar0 > kAlphaMax ? 0.f : a.x, ar1 > kAlphaMax ? 0.f : a.y);
    } else {
        a = make_float2(in0 ? ar0 : 0.f, in1 ? ar1 : 0.f);
        am = a;
    }
    const float2 D = __ffma2_rn(b0, bs.c0p, __ffma2_rn(b1, bs.c1p, __ffma2_rn(b2, bs.c2p, nbF)));
    const float2 oma = __ffma2_rn(a, m1, one2);  // 1 - a
    const float2 inv = make_float2(fast_rcp(oma.x), fast_rcp(oma.y));
    const float2 dLda = __ffma2_rn(Ap, inv, __fmul2_rn(bs.wp, D));
    acc.gw = __ffma2_rn(a, D, acc.gw);
    acc.gc0 = __ffma2_rn(a, b0, acc.gc0);  // times w in the epilogue
    acc.gc1 = __ffma2_rn(a, b1, acc.gc1);
    acc.gc2 = __ffma2_rn(a, b2, acc.gc2);
    const float2 da = __fmul2_rn(dLda, am);
    Rd = __fadd2_rn(Rd, da);
    const float2 qd = __fmul2_rn(da, e1);
    Re = __fadd2_rn(Re, qd);
    acc.See = __ffma2_rn(qd, e1, acc.See);
}

// Rows [rlo, rhi] of the tile for one lane's splat.  kTest: test every pixel
// against the cutoff (the pair contributes iff s <= thr); without it every
// pixel of the rows contributes (the caller knows the whole tile lies inside
// the cutoff ellipse).  A row is taken kQuads groups of four pixels at a
// time: the group's two or four steps run when some lane of the warp has a
// contributing pixel in it (a warp vote, so the branch is uniform), and run
// without branches between them, so that their chains interleave.
template <bool kTest, bool kClamp, int kQuads>
__device__ __forceinline__ void bwd_rows(const BwdSplat &bs, const BwdState &S, int rlo, int rhi, BwdAcc &acc) {
    const float2 zero2 = make_float2(0.f, 0.f);
    for (int ky = rlo; ky <= rhi; ++ky) {
        const RowTerms rt = row_terms(bs.A2dx0, bs.dy0, bs.rA2, bs.B2, ky);
        const float2 e10p = make_float2(rt.e10, rt.e10), e2p = make_float2(rt.e2sq, rt.e2sq);
        float2 Rd = zero2, Re = zero2;
#pragma unroll
        for (int kq0 = 0; kq0 < kTile / 4; kq0 += kQuads) {
            float2 e1[2 * kQuads], sq[2 * kQuads];
            bool in[4 * kQuads];
            bool any = false;
#pragma unroll
            for (int h = 0; h < 2 * kQuads; ++h) {
                const float kx = (float)(4 * kq0 + 2 * h);
                e1[h] = __ffma2_rn(bs.A2p, make_float2(kx, kx + 1.f), e10p);
                sq[h] = __ffma2_rn(e1[h], e1[h], e2p);
                in[2 * h] = !kTest || sq[h].x <= bs.thr;
                in[2 * h + 1] = !kTest || sq[h].y <= bs.thr;
                any = any || in[2 * h] || in[2 * h + 1];
            }
            if (!kTest || __any_sync(0xffffffffu, any)) {
#pragma unroll
                for (int qq = 0; qq < kQuads; ++qq) {
                    const int kq = ky * (kTile / 4) + kq0 + qq;
                    const float4 u0 = S.p[0][kq], u1 = S.p[1][kq], u2 = S.p[2][kq], u3 = S.p[3][kq];
                    const float4 u4 = S.p[4][kq];
                    bwd_step<kClamp>(bs, e1[2 * qq], sq[2 * qq], in[4 * qq], in[4 * qq + 1], make_float2(u0.x, u0.y),
                                     make_float2(u1.x, u1.y), make_float2(u2.x, u2.y), make_float2(u3.x, u3.y),
                                     make_float2(u4.x, u4.y), Rd, Re, acc);
                    bwd_step<kClamp>(bs, e1[2 * qq + 1], sq[2 * qq + 1], in[4 * qq + 2], in[4 * qq + 3],
                                     make_float2(u0.z, u0.w), make_float2(u1.z, u1.w), make_float2(u2.z, u2.w),
                                     make_float2(u3.z, u3.w), make_float2(u4.z, u4.w), Rd, Re, acc);
                }
            }
        }
        const float rd = Rd.x + Rd.y, re = Re.x + Re.y;
        acc.Sd += rd;
        acc.Sdy = fmaf(rd, rt.dy, acc.Sdy);
        acc.Sdyy = fmaf(rd, rt.dy * rt.dy, acc.Sdyy);
        acc.Se += re;
        acc.Sey = fmaf(re, rt.dy, acc.Sey);
    }
}

constexpr int kBwdQuads = 2;  // groups of four pixels per warp vote
// Threads per block (one block per tile).  Each round gives every warp 32 of the tile's splats;
// four warps keep more of a typical tile's warps busy (the median tile holds ~110 splats at a 5 %
// active set) than eight, without stretching the heaviest tiles into long serial chains as two do.
constexpr int kBwdThreads = 128;
constexpr int kBwdMinBlocks = 12 * 64 / kBwdThreads;  // <= 85 registers a thread

template <bool kGroup>
__global__ void __launch_bounds__(kBwdThreads, kBwdMinBlocks) raster_bwd_kernel(const __grid_constant__ Batch b,
                                                              const float4 *__restrict__ rec,
                                                              const int *__restrict__ offsets,
                                                              const uint32_t *__restrict__ pairs, int64_t cap,
                                                              uint32_t nrec, float4 *__restrict__ sgrad) {
    __shared__ BwdState S;
    __shared__ uint32_t sorted[kGroup ? kBwdThreads : 1];
    __shared__ uint8_t sfull[kGroup ? kBwdThreads : 1];
    __shared__ int hist[kBwdKeys];

    const int gt = block_tile(b);
    const int v = find_view(b, gt);
    const ViewDesc &vd = b.v[v];
    const int lt = gt - vd.tile_base;
    const int ty = lt / vd.tiles_x, tx = lt - ty * vd.tiles_x;
    const int tid = threadIdx.x;
#pragma unroll
    for (int t = tid; t < kTilePix; t += kBwdThreads) {
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
    __syncthreads();

    const int start = offsets[gt];
    const int end = (int)min((int64_t)offsets[gt + 1], cap);
    const int warp = tid >> 5, lane = tid & 31;
    const float ox = (float)(tx * kTile) + 0.5f, oy = (float)(ty * kTile) + 0.5f;

    for (int cb0 = start; cb0 < end; cb0 += kBwdThreads) {
        uint32_t q;
        bool full = false;
        if (kGroup) {
            // rank this round's splats: class 0 = the whole tile lies inside the cutoff ellipse (its
            // four corner pixels do, by a margin; the ellipse is convex, so then every pixel does
            // and its rounded exponent stays below the cut), classes 1-16 = the 4x4-pixel cell of
            // the centre (clamped), 17 = no record; then warps take 32 consecutive splats
            const int nr = min(kBwdThreads, end - cb0);
            uint32_t myq = 0xffffffffu;
            int key = kBwdKeys - 1, slot = 0;
            if (tid < kBwdKeys) hist[tid] = 0;
            __syncthreads();
            if (tid < nr) {
                myq = pairs[cb0 + tid];
                if (myq < nrec) {
                    const float4 c0r = rec[3 * (int64_t)myq + 0], c1r = rec[3 * (int64_t)myq + 1];
                    const SplatConsts k = splat_consts(ox, oy, c0r.x, c0r.y, c0r.z, c0r.w, c1r.y);
                    const float lim = k.thr - fmaf(1e-3f, fabsf(k.thr), 1e-3f);
                    bool in = true;
#pragma unroll
                    for (int cyy = 0; cyy < 2; ++cyy) {
                        const RowTerms rt = row_terms(k.A2dx0, k.dy0, k.rA2, c1r.x, cyy * (kTile - 1));
#pragma unroll
                        for (int cxx = 0; cxx < 2; ++cxx)
                            in = in && quad_s(col_e1(c0r.w, rt.e10, cxx * (kTile - 1)), rt.e2sq) <= lim;
                    }
                    const int cx = f2i_clamped(floorf((c0r.x - (ox - 0.5f)) * 0.25f), 0, 3);
                    const int cy = f2i_clamped(floorf((c0r.y - (oy - 0.5f)) * 0.25f), 0, 3);
                    key = in ? 0 : 1 + cy * 4 + cx;
                }
                slot = atomicAdd(&hist[key], 1);
            }
            __syncthreads();
            if (tid == 0) {
                int run = 0;
                for (int c = 0; c < kBwdKeys; ++c) {
                    const int t = hist[c];
                    hist[c] = run;
                    run += t;
                }
            }
            __syncthreads();
            if (tid < nr) {
                sorted[hist[key] + slot] = myq;
                sfull[hist[key] + slot] = key == 0 ? 1 : 0;
            }
            __syncthreads();
            const int idx = warp * 32 + lane;
            q = idx < nr ? sorted[idx] : 0xffffffffu;
            full = idx < nr && sfull[idx] != 0;
            if (cb0 + warp * 32 >= end) continue;  // this warp has no splat in this round
        } else {
            const int idx = cb0 + warp * 32 + lane;
            if (cb0 + warp * 32 >= end) continue;
            q = idx < end ? pairs[idx] : 0xffffffffu;
        }
        const bool valid = q < nrec;
        float4 a0 = make_float4(0.f, 0.f, 0.f, 0.f), a1 = make_float4(0.f, -INFINITY, 0.f, -1.f), a2 = a0;
        if (valid) {
            a0 = rec[3 * (int64_t)q + 0];
            a1 = rec[3 * (int64_t)q + 1];
            a2 = rec[3 * (int64_t)q + 2];
        }
        const float rr = a0.z, A2 = a0.w, B2 = a1.x, log2o = a1.y, w = a1.z, yh = a1.w;
        const SplatConsts sc = splat_consts(ox, oy, a0.x, a0.y, rr, A2, log2o);
        const float dy0 = sc.dy0;
        // rows of the tile this lane's ellipse can reach; the warp walks their union
        int rlo = kTile, rhi = -1;
        if (valid && yh >= 0.f) {
            rlo = f2i_clamped(ceilf(-yh - dy0), 0, kTile);
            rhi = f2i_clamped(floorf(yh - dy0), -1, kTile - 1);
        }
        rlo = __reduce_min_sync(0xffffffffu, rlo);
        rhi = __reduce_max_sync(0xffffffffu, rhi);

        const float2 A2p = make_float2(A2, A2), wp = make_float2(w, w), l2op = make_float2(log2o, log2o);
        const float2 c0p = make_float2(a2.x, a2.x), c1p = make_float2(a2.y, a2.y), c2p = make_float2(a2.z, a2.z);
        const float2 zero2 = make_float2(0.f, 0.f);
        BwdAcc acc;
        acc.See = acc.gw = acc.gc0 = acc.gc1 = acc.gc2 = zero2;
        acc.Se = acc.Sey = acc.Sd = acc.Sdy = acc.Sdyy = 0.f;
        const BwdSplat bs{A2p, wp, l2op, c0p, c1p, c2p, sc.A2dx0, dy0, sc.rA2, B2, sc.thr};
        // a splat with log2 o <= kNoClampLog2 never reaches the 0.99 clamp
        const bool clamp = __any_sync(0xffffffffu, valid && log2o > kNoClampLog2);
        if (kGroup && __all_sync(0xffffffffu, full || !valid)) {  // every pixel of the tile contributes
            if (clamp)
                bwd_rows<false, true, kBwdQuads>(bs, S, 0, kTile - 1, acc);
            else
                bwd_rows<false, false, kBwdQuads>(bs, S, 0, kTile - 1, acc);
        } else if (clamp) {
            bwd_rows<true, true, kBwdQuads>(bs, S, rlo, rhi, acc);
        } else {
            bwd_rows<true, false, kBwdQuads>(bs, S, rlo, rhi, acc);
        }
        const float Se = acc.Se, Sey = acc.Sey, Sd = acc.Sd, Sdy = acc.Sdy, Sdyy = acc.Sdyy;
        const float2 See = acc.See, gw = acc.gw, gc0 = acc.gc0, gc1 = acc.gc1, gc2 = acc.gc2;
        if (valid) {
            const float K = -2.f * kLn2;
            const float See1 = See.x + See.y;
            const float g_mx = -K * A2 * Se;
            const float g_my = K * (A2 * rr * Se - B2 * B2 * Sdy);
            const float g_r = -K * A2 * Sey;
            const float g_A2 = K * See1 / A2;
            const float g_B2 = K * B2 * Sdyy;
            float4 *out = sgrad + 3 * (int64_t)q;
            atomicAdd(out + 0, make_float4(g_mx, g_my, g_r, g_A2));
            atomicAdd(out + 1, make_float4(g_B2, Sd, gw.x + gw.y, w * (gc0.x + gc0.y)));
            atomicAdd(reinterpret_cast<float2 *>(out + 2), make_float2(w * (gc1.x + gc1.y), w * (gc2.x + gc2.y)));
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

int launch_raster_bwd(const Batch &b, bool group, const float4 *rec, const int *offsets, const uint32_t *pairs,
                      int64_t cap, float4 *sgrad, cudaStream_t st) {
    if (b.total_tiles == 0) return 0;
    const uint32_t nrec = (uint32_t)((int64_t)b.n_views * b.n_list);
    if (group)
        raster_bwd_kernel<true><<<b.total_tiles, kBwdThreads, 0, st>>>(b, rec, offsets, pairs, cap, nrec, sgrad);
    else
        raster_bwd_kernel<false><<<b.total_tiles, kBwdThreads, 0, st>>>(b, rec, offsets, pairs, cap, nrec, sgrad);
    return 0;
}

}  // namespace soit
