// raster_fwd.cu -- tile rasteriser of the OIT sums (Alg. 2 BAN / BAU, Eq. 7).
//
// One thread block per 16x16 tile of the batch, one thread per pixel.  The
// tile's records are staged through shared memory 256 at a time; every
// thread accumulates, over the tile's splats, P += a w c, Q += a w and
// T *= (1 - a) (per-batch partial sums for P and Q to hold the FP32
// rounding of long sums).  The epilogue depends on the mode:
//   kRasterFused: combine with the view's frozen sums (P_F, Q_F, log T_F),
//     write C = T c0 + (1 - T) P/Q, the L1 loss and the backward pixel state
//     (g, A = T g.(F - c0), B = (1 - T)/Q, g.F) with g = sign(C - I)/(3HW).
//   kRasterAux: as fused but without a target; writes (F, T, Q) for the
//     backward to turn into the state once dL/dC is known.
//   kRasterSums: the records carry a sign s = +-1; adds s a w c, s a w and
//     s log(1 - a) to the frozen planes (the delayed pre-render update).
#include "common.cuh"
#include "launch.h"

namespace soit {

template <int kMode>
__global__ void __launch_bounds__(kTilePix) raster_fwd_kernel(const __grid_constant__ Batch b,
                                                              const float4 *__restrict__ rec,
                                                              const int *__restrict__ offsets,
                                                              const uint32_t *__restrict__ pairs, int64_t cap, uint32_t nrec,
                                                              float bg0, float bg1, float bg2, float *loss,
                                                              unsigned long long *contrib) {
    __shared__ float4 s0[kTilePix], s1[kTilePix], s2[kTilePix];
    __shared__ float red[kTilePix / 32];
    __shared__ unsigned red_n[kTilePix / 32];

    const int gt = blockIdx.x;
    const int v = find_view(b, gt);
    const ViewDesc &vd = b.v[v];
    const int lt = gt - vd.tile_base;
    const int ty = lt / vd.tiles_x, tx = lt - ty * vd.tiles_x;
    const int tid = threadIdx.x;
    const int x = tx * kTile + (tid & (kTile - 1)), y = ty * kTile + (tid >> 4);
    const bool inside = x < vd.W && y < vd.H;
    const float px = (float)x + 0.5f, py = (float)y + 0.5f;

    const int start = offsets[gt];
    const int end = (int)min((int64_t)offsets[gt + 1], cap);

    float P0 = 0.f, P1 = 0.f, P2 = 0.f, Q = 0.f, T = 1.f, LT = 0.f;
    unsigned n_contrib = 0;
    for (int base = start; base < end; base += kTilePix) {
        const int n = min(kTilePix, end - base);
        __syncthreads();
        if (tid < n) {
            const uint32_t q = pairs[base + tid];
            if (q < nrec) {
                s0[tid] = rec[3 * (int64_t)q + 0];
                s1[tid] = rec[3 * (int64_t)q + 1];
                s2[tid] = rec[3 * (int64_t)q + 2];
            } else {  // never written by this call's scatter: contributes nothing
                s0[tid] = make_float4(0.f, 0.f, 0.f, 0.f);
                s1[tid] = make_float4(0.f, -INFINITY, 0.f, 0.f);
                s2[tid] = make_float4(0.f, 0.f, 0.f, 0.f);
            }
        }
        __syncthreads();
        float b0 = 0.f, b1 = 0.f, b2 = 0.f, bq = 0.f, bl = 0.f;
        for (int j = 0; j < n; ++j) {
            const float4 a0 = s0[j], a1 = s1[j];
            const float dx = px - a0.x, dy = py - a0.y;
            const float u = fmaf(-a0.z, dy, dx);
            const float e1 = a0.w * u, e2 = a1.x * dy;
            const float arg = a1.y - fmaf(e1, e1, e2 * e2);
            if (arg >= -kLog2_255) {
                const float a = fminf(exp2f(arg), kAlphaMax);
                const float4 a2 = s2[j];
                float aw = a * a1.z;
                if (kMode == kRasterSums) aw *= a2.z;
                b0 = fmaf(aw, a1.w, b0);
                b1 = fmaf(aw, a2.x, b1);
                b2 = fmaf(aw, a2.y, b2);
                bq += aw;
                if (kMode == kRasterSums)
                    bl = fmaf(a2.z, log1pf(-a), bl);
                else
                    T = fmaf(-T, a, T);
                ++n_contrib;
            }
        }
        P0 += b0; P1 += b1; P2 += b2; Q += bq; LT += bl;
    }

    const int64_t HW = (int64_t)vd.W * vd.H;
    const int64_t pix = (int64_t)y * vd.W + x;
    float my_loss = 0.f;
    if (inside) {
        if (kMode == kRasterSums) {
            float *fz = vd.frozen;
            fz[pix] += P0;
            fz[HW + pix] += P1;
            fz[2 * HW + pix] += P2;
            fz[3 * HW + pix] += Q;
            fz[4 * HW + pix] += LT;
        } else {
            const float *fz = vd.frozen;
            const float Pt0 = P0 + fz[pix], Pt1 = P1 + fz[HW + pix], Pt2 = P2 + fz[2 * HW + pix];
            const float Qt = Q + fz[3 * HW + pix];
            const float Tt = T * expf(fz[4 * HW + pix]);
            const float invQ = Qt > 0.f ? 1.f / Qt : 0.f;
            const float F0 = Pt0 * invQ, F1 = Pt1 * invQ, F2 = Pt2 * invQ;
            const float omT = 1.f - Tt;
            const float C0 = fmaf(Tt, bg0, omT * F0), C1 = fmaf(Tt, bg1, omT * F1), C2 = fmaf(Tt, bg2, omT * F2);
            float *img = vd.image + 3 * pix;
            img[0] = C0; img[1] = C1; img[2] = C2;
            float *st = vd.state;
            if (kMode == kRasterFused) {
                const float *tg = vd.target + 3 * pix;
                const float d0 = C0 - tg[0], d1 = C1 - tg[1], d2 = C2 - tg[2];
                my_loss = fabsf(d0) + fabsf(d1) + fabsf(d2);
                const float inv = 1.f / (3.f * (float)HW);
                const float g0 = d0 > 0.f ? inv : (d0 < 0.f ? -inv : 0.f);
                const float g1 = d1 > 0.f ? inv : (d1 < 0.f ? -inv : 0.f);
                const float g2 = d2 > 0.f ? inv : (d2 < 0.f ? -inv : 0.f);
                st[pix] = g0;
                st[HW + pix] = g1;
                st[2 * HW + pix] = g2;
                st[3 * HW + pix] = Tt * (g0 * (F0 - bg0) + g1 * (F1 - bg1) + g2 * (F2 - bg2));
                st[4 * HW + pix] = omT * invQ;
                st[5 * HW + pix] = g0 * F0 + g1 * F1 + g2 * F2;
            } else {
                st[pix] = F0;
                st[HW + pix] = F1;
                st[2 * HW + pix] = F2;
                st[3 * HW + pix] = Tt;
                st[4 * HW + pix] = Qt;
            }
        }
    } else {
        n_contrib = 0;
    }
    if ((kMode == kRasterFused && loss) || contrib) {
        float l = my_loss;
        unsigned c = n_contrib;
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            l += __shfl_xor_sync(0xffffffffu, l, off);
            c += __shfl_xor_sync(0xffffffffu, c, off);
        }
        if ((tid & 31) == 0) { red[tid >> 5] = l; red_n[tid >> 5] = c; }
        __syncthreads();
        if (tid == 0) {
            float ls = 0.f;
            unsigned long long cs = 0;
            for (int k = 0; k < kTilePix / 32; ++k) { ls += red[k]; cs += red_n[k]; }
            if (kMode == kRasterFused && loss && ls != 0.f) atomicAdd(loss, ls / (3.f * (float)HW));
            if (contrib && cs) atomicAdd(contrib, cs);
        }
    }
}

int launch_raster_fwd(const Batch &b, int mode, const float4 *rec, const int *offsets, const uint32_t *pairs,
                      int64_t cap, const float bg[3], float *loss, unsigned long long *contrib, cudaStream_t st) {
    const uint32_t nrec = (uint32_t)((int64_t)b.n_views * b.n_list);
    if (b.total_tiles == 0) return 0;
    const dim3 grid(b.total_tiles);
    switch (mode) {
        case kRasterFused:
            raster_fwd_kernel<kRasterFused><<<grid, kTilePix, 0, st>>>(b, rec, offsets, pairs, cap, nrec, bg[0], bg[1],
                                                                      bg[2], loss, contrib);
            break;
        case kRasterAux:
            raster_fwd_kernel<kRasterAux><<<grid, kTilePix, 0, st>>>(b, rec, offsets, pairs, cap, nrec, bg[0], bg[1], bg[2],
                                                                    loss, contrib);
            break;
        default:
            raster_fwd_kernel<kRasterSums><<<grid, kTilePix, 0, st>>>(b, rec, offsets, pairs, cap, nrec, bg[0], bg[1],
                                                                     bg[2], loss, contrib);
            break;
    }
    return 0;
}

}  // namespace soit
