// ssim.cu -- the 3DGS photometric loss L = (1 - lambda) L1 + lambda (1 - SSIM)
// (Sec. 5.1: the paper keeps the loss of the original 3DGS) and its image
// gradient, turned directly into the backward raster's pixel state.
//
// SSIM per colour channel with an 11 x 11 Gaussian window (sigma 1.5), zero
// padding outside the image, C1 = 0.01^2, C2 = 0.03^2, averaged over pixels
// and channels.  With mu = G * x, E[xx] = G * x^2, E[xy] = G * (x y) and
// S = (2 mu_x mu_y + C1)(2 s_xy + C2) / ((mu_x^2 + mu_y^2 + C1)(s_xx + s_yy + C2)),
// the gradient of sum(S) is G * a + 2 x (G * b) + y (G * c) with, per output
// pixel, a = dS/dmu_x, b = dS/dE[xx], c = dS/dE[xy] (the window is symmetric,
// so the adjoint of the zero-padded filter is the same filter).
//
// Two passes per view, both on 32 x 16 output tiles with a 5-pixel halo held
// in shared memory and the separable window applied rows first:
//   ssim_fwd_kernel (all channels per block): the five filtered moments, S and
//     (a, b, c) per pixel and channel, written as [3 channels][H, W, 3]; block
//     sums of S and |x - y| into per-view doubles;
//   ssim_bwd_kernel (all channels per block): filters (a, b, c), forms
//     dL/dC and rewrites the forward's (F, T, Q) planes into the pixel state
//     (B g, A, -B g.F) that the backward raster reads.
#include "common.cuh"
#include "launch.h"

namespace soit {

constexpr int kSsimTW = 32, kSsimTH = 16, kSsimR = 5, kSsimK = 2 * kSsimR + 1;
constexpr int kSsimHW = kSsimTW + 2 * kSsimR, kSsimHH = kSsimTH + 2 * kSsimR;  // 42 x 26 halo tile
constexpr float kSsimC1 = 0.01f * 0.01f, kSsimC2 = 0.03f * 0.03f;

// One block per 32 x 16 tile, all three channels: the image and target halo
// tiles are read once (interleaved, coalesced) into (x, y) pairs.  Per
// channel, rows first: a thread filters 4 adjacent outputs of one halo row
// from 14 inputs held in registers, the (x, y) and (x^2, y^2) moments as
// f32x2 pairs; then columns: a thread filters 2 adjacent output rows of one
// column from 12 staged rows.  S and the partials (a, b, c) per pixel and
// channel are written as abc = [3 channels][H, W, 3] (each channel's pass of
// the backward then reads one contiguous array).
__global__ void __launch_bounds__(256) ssim_fwd_kernel(const float *__restrict__ img, const float *__restrict__ tgt,
                                                       int W, int H, SsimWindow win, float *__restrict__ abc,
                                                       double *__restrict__ sums) {
    __shared__ float2 xy[3][kSsimHH][kSsimHW];           // (x, y) per channel
    __shared__ float2 hm[2][kSsimHH][kSsimTW];           // filtered rows: (x, y), (x^2, y^2)
    __shared__ float hc[kSsimHH][kSsimTW];               // filtered rows: x y
    __shared__ float red[2][8];
    const int x0 = blockIdx.x * kSsimTW, y0 = blockIdx.y * kSsimTH;
    const int tid = threadIdx.x, tx = tid & 31, ty = tid >> 5;
    for (int i = tid; i < kSsimHH * kSsimHW * 3; i += blockDim.x) {
        const int r = i / (kSsimHW * 3), e = i - r * (kSsimHW * 3);
        const int c = e / 3, ch = e - c * 3;
        const int gy = y0 - kSsimR + r, gx = x0 - kSsimR + c;
        const bool in = gx >= 0 && gx < W && gy >= 0 && gy < H;
        const int64_t o = ((int64_t)gy * W + gx) * 3 + ch;
        xy[ch][r][c] = make_float2(in ? img[o] : 0.f, in ? tgt[o] : 0.f);
    }
    float s_sum = 0.f, l1_sum = 0.f;
    for (int ch = 0; ch < 3; ++ch) {
        __syncthreads();
        if (tid < kSsimHH * (kSsimTW / 4)) {  // 26 rows x 8 groups of 4 outputs
            const int r = tid >> 3, c0 = (tid & 7) * 4;
            float2 v[kSsimK + 3], v2[kSsimK + 3];
            float vp[kSsimK + 3];
#pragma unroll
            for (int j = 0; j < kSsimK + 3; ++j) {
                v[j] = xy[ch][r][c0 + j];
                v2[j] = __fmul2_rn(v[j], v[j]);
                vp[j] = v[j].x * v[j].y;
            }
#pragma unroll
            for (int o = 0; o < 4; ++o) {
                float2 m1 = make_float2(0.f, 0.f), m2 = m1;
                float mp = 0.f;
#pragma unroll
                for (int k = 0; k < kSsimK; ++k) {
                    const float2 wk = make_float2(win.w[k], win.w[k]);
                    m1 = __ffma2_rn(wk, v[o + k], m1);
                    m2 = __ffma2_rn(wk, v2[o + k], m2);
                    mp = fmaf(win.w[k], vp[o + k], mp);
                }
                hm[0][r][c0 + o] = m1;
                hm[1][r][c0 + o] = m2;
                hc[r][c0 + o] = mp;
            }
        }
        __syncthreads();
        {
            const int rr0 = ty * 2;  // two output rows per thread: 8 x 2 = 16
            float2 a1[2] = {make_float2(0.f, 0.f), make_float2(0.f, 0.f)}, a2[2] = {a1[0], a1[0]};
            float ap[2] = {0.f, 0.f};
#pragma unroll
            for (int j = 0; j < kSsimK + 1; ++j) {
                const float2 h1 = hm[0][rr0 + j][tx], h2 = hm[1][rr0 + j][tx];
                const float hp = hc[rr0 + j][tx];
#pragma unroll
                for (int o = 0; o < 2; ++o) {
                    const int k = j - o;
                    if (k < 0 || k >= kSsimK) continue;
                    const float2 wk = make_float2(win.w[k], win.w[k]);
                    a1[o] = __ffma2_rn(wk, h1, a1[o]);
                    a2[o] = __ffma2_rn(wk, h2, a2[o]);
                    ap[o] = fmaf(win.w[k], hp, ap[o]);
                }
            }
#pragma unroll
            for (int o = 0; o < 2; ++o) {
                const int gx = x0 + tx, gy = y0 + rr0 + o;
                if (gx >= W || gy >= H) continue;
                const float mx = a1[o].x, my = a1[o].y;
                const float sxx = a2[o].x - mx * mx, syy = a2[o].y - my * my, sxy = ap[o] - mx * my;
                const float A = 2.f * mx * my + kSsimC1, B = 2.f * sxy + kSsimC2;
                const float Cc = mx * mx + my * my + kSsimC1, D = sxx + syy + kSsimC2;
                const float S = (A * B) / (Cc * D);
                float *out = abc + (ch * (int64_t)W * H + (int64_t)gy * W + gx) * 3;
                out[0] = S * (2.f * my / A - 2.f * my / B - 2.f * mx / Cc + 2.f * mx / D);  // dS/dmu_x
                out[1] = -S / D;                                                              // dS/dE[xx]
                out[2] = 2.f * S / B;                                                         // dS/dE[xy]
                s_sum += S;
                const float2 c = xy[ch][rr0 + o + kSsimR][tx + kSsimR];
                l1_sum += fabsf(c.x - c.y);
            }
        }
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        s_sum += __shfl_xor_sync(0xffffffffu, s_sum, off);
        l1_sum += __shfl_xor_sync(0xffffffffu, l1_sum, off);
    }
    if (tx == 0) {
        red[0][ty] = s_sum;
        red[1][ty] = l1_sum;
    }
    __syncthreads();
    if (tid == 0) {
        double sv = 0.0, lv = 0.0;
        for (int k = 0; k < 8; ++k) {
            sv += red[0][k];
            lv += red[1][k];
        }
        atomicAdd(sums + 0, sv);
        atomicAdd(sums + 1, lv);
    }
}

// One block per 32 x 16 tile: per channel, the (a, b, c) halo tile is read
// once (interleaved) and filtered rows first (4 outputs per thread from 14
// register-held inputs), then columns (2 output rows per thread); dL/dC per
// pixel, then the state rewrite.
__global__ void __launch_bounds__(256) ssim_bwd_kernel(const float *__restrict__ img, const float *__restrict__ tgt,
                                                       int W, int H, SsimWindow win, const float *__restrict__ abc,
                                                       float lambda, float bg0, float bg1, float bg2,
                                                       float *__restrict__ state, float *__restrict__ grad_out) {
    __shared__ float2 mab[kSsimHH][kSsimHW];       // (a, b) of one channel
    __shared__ float mc[kSsimHH][kSsimHW];         // c of one channel
    __shared__ float2 hab[3][kSsimHH][kSsimTW];    // filtered rows (a, b) per channel
    __shared__ float hcc[3][kSsimHH][kSsimTW];     // filtered rows c per channel
    const int x0 = blockIdx.x * kSsimTW, y0 = blockIdx.y * kSsimTH;
    const int tid = threadIdx.x, tx = tid & 31, ty = tid >> 5;
    const int64_t HW = (int64_t)W * H;
    for (int ch = 0; ch < 3; ++ch) {
        __syncthreads();
        for (int i = tid; i < kSsimHH * kSsimHW; i += blockDim.x) {
            const int r = i / kSsimHW, c = i - r * kSsimHW;
            const int gy = y0 - kSsimR + r, gx = x0 - kSsimR + c;
            float2 v = make_float2(0.f, 0.f);
            float vc = 0.f;
            if (gx >= 0 && gx < W && gy >= 0 && gy < H) {
                const float *p = abc + (ch * HW + (int64_t)gy * W + gx) * 3;
                v = make_float2(p[0], p[1]);
                vc = p[2];
            }
            mab[r][c] = v;
            mc[r][c] = vc;
        }
        __syncthreads();
        if (tid < kSsimHH * (kSsimTW / 4)) {
            const int r = tid >> 3, c0 = (tid & 7) * 4;
            float2 v[kSsimK + 3];
            float vc[kSsimK + 3];
#pragma unroll
            for (int j = 0; j < kSsimK + 3; ++j) {
                v[j] = mab[r][c0 + j];
                vc[j] = mc[r][c0 + j];
            }
#pragma unroll
            for (int o = 0; o < 4; ++o) {
                float2 ab = make_float2(0.f, 0.f);
                float cc = 0.f;
#pragma unroll
                for (int k = 0; k < kSsimK; ++k) {
                    ab = __ffma2_rn(make_float2(win.w[k], win.w[k]), v[o + k], ab);
                    cc = fmaf(win.w[k], vc[o + k], cc);
                }
                hab[ch][r][c0 + o] = ab;
                hcc[ch][r][c0 + o] = cc;
            }
        }
    }
    __syncthreads();
    const float inv_n = 1.f / (3.f * (float)HW);
    const int rr0 = ty * 2;
    float g[2][3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        float2 ab[2] = {make_float2(0.f, 0.f), make_float2(0.f, 0.f)};
        float cc[2] = {0.f, 0.f};
#pragma unroll
        for (int j = 0; j < kSsimK + 1; ++j) {
            const float2 h = hab[c][rr0 + j][tx];
            const float hz = hcc[c][rr0 + j][tx];
#pragma unroll
            for (int o = 0; o < 2; ++o) {
                const int k = j - o;
                if (k < 0 || k >= kSsimK) continue;
                ab[o] = __ffma2_rn(make_float2(win.w[k], win.w[k]), h, ab[o]);
                cc[o] = fmaf(win.w[k], hz, cc[o]);
            }
        }
#pragma unroll
        for (int o = 0; o < 2; ++o) {
            const int gx = x0 + tx, gy = y0 + rr0 + o;
            g[o][c] = 0.f;
            if (gx >= W || gy >= H) continue;
            const int64_t pix = (int64_t)gy * W + gx;
            const float x = img[3 * pix + c], y = tgt[3 * pix + c];
            const float dS = ab[o].x + 2.f * x * ab[o].y + y * cc[o];
            const float d = x - y;
            const float sg = d > 0.f ? 1.f : (d < 0.f ? -1.f : 0.f);
            g[o][c] = ((1.f - lambda) * sg - lambda * dS) * inv_n;
            if (grad_out) grad_out[3 * pix + c] = g[o][c];
        }
    }
#pragma unroll
    for (int o = 0; o < 2; ++o) {
        const int gx = x0 + tx, gy = y0 + rr0 + o;
        if (gx >= W || gy >= H) continue;
        const int64_t pix = (int64_t)gy * W + gx;
        // the forward left F (3), T, Q in the state planes; turn them into the backward state
        const float F0 = state[pix], F1 = state[HW + pix], F2 = state[2 * HW + pix];
        const float T = state[3 * HW + pix], Q = state[4 * HW + pix];
        const float Bq = Q > 0.f ? (1.f - T) / Q : 0.f;
        const float *gg = g[o];
        state[pix] = Bq * gg[0];
        state[HW + pix] = Bq * gg[1];
        state[2 * HW + pix] = Bq * gg[2];
        state[3 * HW + pix] = T * (gg[0] * (F0 - bg0) + gg[1] * (F1 - bg1) + gg[2] * (F2 - bg2));
        state[4 * HW + pix] = -Bq * (gg[0] * F0 + gg[1] * F1 + gg[2] * F2);
    }
}

// sums[2 v] = sum of S, sums[2 v + 1] = sum |x - y| of view v; loss = sum over views of
// (1 - lambda) mean|x - y| + lambda (1 - mean S).
__global__ void ssim_loss_kernel(const double *__restrict__ sums, const __grid_constant__ SsimLossArgs a,
                                 float *loss) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    double l = 0.0;
    for (int v = 0; v < a.n_views; ++v)
        l += (1.0 - a.lambda) * sums[2 * v + 1] * a.inv_n[v] + a.lambda * (1.0 - sums[2 * v] * a.inv_n[v]);
    *loss = (float)l;
}

int launch_ssim_view(const float *img, const float *tgt, int W, int H, const SsimWindow &win, float *abc,
                     double *sums, float lambda, const float bg[3], float *state, float *grad_out, cudaStream_t st) {
    const dim3 grid((W + kSsimTW - 1) / kSsimTW, (H + kSsimTH - 1) / kSsimTH, 1);
    ssim_fwd_kernel<<<grid, 256, 0, st>>>(img, tgt, W, H, win, abc, sums);
    ssim_bwd_kernel<<<grid, 256, 0, st>>>(img, tgt, W, H, win, abc, lambda, bg[0], bg[1], bg[2], state, grad_out);
    return 0;
}

int launch_ssim_loss(const double *sums, const SsimLossArgs &a, float *loss, cudaStream_t st) {
    ssim_loss_kernel<<<1, 32, 0, st>>>(sums, a, loss);
    return 0;
}

}  // namespace soit
