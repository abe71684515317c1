// raster_bwd.cu -- backward of the OIT raster (App. B, Eq. 9-10; Sec. 4.2).
//
// Per-splat parallel: a tile's 256 pixel states are loaded into shared
// memory once; each warp takes 32 of the tile's splats (lane = splat) and
// walks all 256 pixels, reading each pixel's state as a shared-memory
// broadcast.  Nothing is stored per pixel in the forward except the state,
// the per-pair alpha is recomputed from the same record, and each lane ends
// the tile with its splat's full tile gradient in registers, added with one
// vector atomic per 4 fields.  No pair is evaluated twice.
//
// Per pixel state (g = dL/dC): A = T g.(F - c0), B = (1 - T)/Q (0 if Q = 0),
// gF = g.F.  Eq. 10 contracted with g gives, per pair,
//   dL/da = A/(1 - a) + B w (g.c - gF),  dL/dw = B a (g.c - gF),
//   dL/dc = B a w g,
// and, unless a is clamped at 0.99, with a = 2^(log2 o - s),
// s = (A2 u)^2 + (B2 dy)^2, u = dx - r dy:  dL/d(ln o) = a dL/da and
// dL/ds = -ln2 a dL/da, chained to (mu'x, mu'y, r, A2, B2).
#include "common.cuh"
#include "launch.h"

namespace soit {

__global__ void __launch_bounds__(kTilePix) raster_bwd_kernel(const __grid_constant__ Batch b,
                                                              const float4 *__restrict__ rec,
                                                              const int *__restrict__ offsets,
                                                              const uint32_t *__restrict__ pairs, int64_t cap, uint32_t nrec,
                                                              float4 *__restrict__ sgrad) {
    __shared__ float4 sa[kTilePix];  // g0, g1, g2, A
    __shared__ float2 sb[kTilePix];  // B, gF

    const int gt = blockIdx.x;
    const int v = find_view(b, gt);
    const ViewDesc &vd = b.v[v];
    const int lt = gt - vd.tile_base;
    const int ty = lt / vd.tiles_x, tx = lt - ty * vd.tiles_x;
    const int tid = threadIdx.x;
    {
        const int x = tx * kTile + (tid & (kTile - 1)), y = ty * kTile + (tid >> 4);
        float4 a = make_float4(0.f, 0.f, 0.f, 0.f);
        float2 c = make_float2(0.f, 0.f);
        if (x < vd.W && y < vd.H) {
            const int64_t HW = (int64_t)vd.W * vd.H, pix = (int64_t)y * vd.W + x;
            const float *st = vd.state;
            a = make_float4(st[pix], st[HW + pix], st[2 * HW + pix], st[3 * HW + pix]);
            c = make_float2(st[4 * HW + pix], st[5 * HW + pix]);
        }
        sa[tid] = a;
        sb[tid] = c;
    }
    __syncthreads();

    const int start = offsets[gt];
    const int end = (int)min((int64_t)offsets[gt + 1], cap);
    const int warp = tid >> 5, lane = tid & 31;
    const float ox = (float)(tx * kTile) + 0.5f, oy = (float)(ty * kTile) + 0.5f;

    for (int cb = start + warp * 32; cb < end; cb += kTilePix) {
        const int idx = cb + lane;
        uint32_t q = idx < end ? pairs[idx] : 0xffffffffu;
        const bool valid = q < nrec;
        float4 a0 = make_float4(0.f, 0.f, 0.f, 0.f), a1 = make_float4(0.f, -INFINITY, 0.f, 0.f), a2 = a0;
        if (valid) {
            a0 = rec[3 * (int64_t)q + 0];
            a1 = rec[3 * (int64_t)q + 1];
            a2 = rec[3 * (int64_t)q + 2];
        }
        const float rr = a0.z, A2 = a0.w, B2 = a1.x, log2o = a1.y, w = a1.z;
        const float c0 = a1.w, c1 = a2.x, c2 = a2.y;
        float S1 = 0.f, S2 = 0.f, S3 = 0.f, S4 = 0.f, S5 = 0.f, gl = 0.f, gw = 0.f;
        float gc0 = 0.f, gc1 = 0.f, gc2 = 0.f;
        const float dx0 = ox - a0.x, dy0 = oy - a0.y;
        for (int ky = 0; ky < kTile; ++ky) {
            const float dy = dy0 + (float)ky;
            const float e2 = B2 * dy;
            const float e2sq = e2 * e2;
#pragma unroll 4
            for (int kx = 0; kx < kTile; ++kx) {
                const float dx = dx0 + (float)kx;
                const float u = fmaf(-rr, dy, dx);
                const float e1 = A2 * u;
                const float arg = log2o - fmaf(e1, e1, e2sq);
                if (arg >= -kLog2_255) {
                    const int k = ky * kTile + kx;
                    const float4 p = sa[k];
                    const float2 pb = sb[k];
                    const float ar = exp2f(arg);
                    const float a = fminf(ar, kAlphaMax);
                    const float gcd = fmaf(p.x, c0, fmaf(p.y, c1, p.z * c2)) - pb.y;  // g.c - gF
                    const float Bg = pb.x * gcd;
                    const float dLda = fmaf(p.w, 1.f / (1.f - a), w * Bg);
                    gw = fmaf(a, Bg, gw);
                    const float Baw = pb.x * a * w;
                    gc0 = fmaf(Baw, p.x, gc0);
                    gc1 = fmaf(Baw, p.y, gc1);
                    gc2 = fmaf(Baw, p.z, gc2);
                    const float da = ar <= kAlphaMax ? dLda * a : 0.f;
                    gl += da;
                    const float G2 = -2.f * kLn2 * da;  // 2 dL/ds
                    const float t = G2 * e1;
                    S1 += t;
                    S2 = fmaf(t, dy, S2);
                    S3 = fmaf(t, u, S3);
                    const float h = G2 * e2;
                    S4 += h;
                    S5 = fmaf(h, dy, S5);
                }
            }
        }
        if (valid) {
            // s = (A2 u)^2 + (B2 dy)^2, u = (px - mx) - r (py - my), dy = py - my
            const float g_mx = -A2 * S1;
            const float g_my = A2 * rr * S1 - B2 * S4;
            const float g_r = -A2 * S2;
            const float g_A2 = S3;
            const float g_B2 = S5;
            float4 *out = sgrad + 3 * (int64_t)q;
            atomicAdd(out + 0, make_float4(g_mx, g_my, g_r, g_A2));
            atomicAdd(out + 1, make_float4(g_B2, gl, gw, gc0));
            atomicAdd(reinterpret_cast<float2 *>(out + 2), make_float2(gc1, gc2));
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
        st[pix] = g0;
        st[HW + pix] = g1;
        st[2 * HW + pix] = g2;
        st[3 * HW + pix] = T * (g0 * (F0 - bg0) + g1 * (F1 - bg1) + g2 * (F2 - bg2));
        st[4 * HW + pix] = Q > 0.f ? (1.f - T) / Q : 0.f;
        st[5 * HW + pix] = g0 * F0 + g1 * F1 + g2 * F2;
    }
}

int launch_prep_state(const Batch &b, const float bg[3], cudaStream_t st) {
    prep_state_kernel<<<dim3(304, b.n_views), 256, 0, st>>>(b, bg[0], bg[1], bg[2]);
    return 0;
}

int launch_raster_bwd(const Batch &b, const float4 *rec, const int *offsets, const uint32_t *pairs, int64_t cap,
                      float4 *sgrad, cudaStream_t st) {
    if (b.total_tiles == 0) return 0;
    const uint32_t nrec = (uint32_t)((int64_t)b.n_views * b.n_list);
    raster_bwd_kernel<<<b.total_tiles, kTilePix, 0, st>>>(b, rec, offsets, pairs, cap, nrec, sgrad);
    return 0;
}

}  // namespace soit
