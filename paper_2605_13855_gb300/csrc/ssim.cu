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
//     (a, b, c) per pixel and channel, written interleaved [H, W, 9]; block
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

// Loads the halo tile of C interleaved values per pixel (rows of (42 C)
// contiguous floats of a [H, W, C] image, coalesced) into dst[r][c * C + j],
// zeros outside the image.
template <int C>
__device__ __forceinline__ void load_halo(float *__restrict__ dst, const float *__restrict__ src, int x0, int y0, int W,
                                          int H) {
    constexpr int RW = kSsimHW * C;
    for (int i = threadIdx.x; i < kSsimHH * RW; i += blockDim.x) {
        const int r = i / RW, e = i - r * RW;
        const int gy = y0 - kSsimR + r, gx = x0 - kSsimR + e / C;
        dst[i] = (gx >= 0 && gx < W && gy >= 0 && gy < H) ? src[((int64_t)gy * W + gx) * C + (e % C)] : 0.f;
    }
}

// One block per 32 x 16 tile, all three channels: the image and target halo
// tiles are read once (interleaved, coalesced); per channel the five moments
// are filtered (rows, then columns) and S, a, b, c formed.  abc: [H, W, 9]
// (a, b, c of channel 0, then 1, then 2).
__global__ void __launch_bounds__(256) ssim_fwd_kernel(const float *__restrict__ img, const float *__restrict__ tgt,
                                                       int W, int H, SsimWindow win, float *__restrict__ abc,
                                                       double *__restrict__ sums) {
    __shared__ float xs[kSsimHH * kSsimHW * 3], ys[kSsimHH * kSsimHW * 3];
    __shared__ float hs[5][kSsimHH][kSsimTW];
    __shared__ float red[2][8];
    const int x0 = blockIdx.x * kSsimTW, y0 = blockIdx.y * kSsimTH;
    const int tid = threadIdx.x, tx = tid & 31, ty = tid >> 5;
    load_halo<3>(xs, img, x0, y0, W, H);
    load_halo<3>(ys, tgt, x0, y0, W, H);
    float s_sum = 0.f, l1_sum = 0.f;
    for (int ch = 0; ch < 3; ++ch) {
        __syncthreads();
        for (int i = tid; i < kSsimHH * kSsimTW; i += blockDim.x) {
            const int r = i / kSsimTW, c = i - r * kSsimTW;
            const float *xr = xs + (r * kSsimHW + c) * 3 + ch, *yr = ys + (r * kSsimHW + c) * 3 + ch;
            float sx = 0.f, sy = 0.f, sxx = 0.f, syy = 0.f, sxy = 0.f;
#pragma unroll
            for (int k = 0; k < kSsimK; ++k) {
                const float w = win.w[k], xv = xr[3 * k], yv = yr[3 * k];
                sx = fmaf(w, xv, sx);
                sy = fmaf(w, yv, sy);
                sxx = fmaf(w, xv * xv, sxx);
                syy = fmaf(w, yv * yv, syy);
                sxy = fmaf(w, xv * yv, sxy);
            }
            hs[0][r][c] = sx;
            hs[1][r][c] = sy;
            hs[2][r][c] = sxx;
            hs[3][r][c] = syy;
            hs[4][r][c] = sxy;
        }
        __syncthreads();
        for (int rr = ty; rr < kSsimTH; rr += 8) {
            const int gx = x0 + tx, gy = y0 + rr;
            if (gx >= W || gy >= H) continue;
            float m[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
#pragma unroll
            for (int k = 0; k < kSsimK; ++k)
#pragma unroll
                for (int q = 0; q < 5; ++q) m[q] = fmaf(win.w[k], hs[q][rr + k][tx], m[q]);
            const float mx = m[0], my = m[1];
            const float sxx = m[2] - mx * mx, syy = m[3] - my * my, sxy = m[4] - mx * my;
            const float A = 2.f * mx * my + kSsimC1, B = 2.f * sxy + kSsimC2;
            const float Cc = mx * mx + my * my + kSsimC1, D = sxx + syy + kSsimC2;
            const float S = (A * B) / (Cc * D);
            float *o = abc + ((int64_t)gy * W + gx) * 9 + 3 * ch;
            o[0] = S * (2.f * my / A - 2.f * my / B - 2.f * mx / Cc + 2.f * mx / D);  // dS/dmu_x
            o[1] = -S / D;                                                              // dS/dE[xx]
            o[2] = 2.f * S / B;                                                         // dS/dE[xy]
            s_sum += S;
            const int ci = ((rr + kSsimR) * kSsimHW + tx + kSsimR) * 3 + ch;
            l1_sum += fabsf(xs[ci] - ys[ci]);
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
// once (interleaved) and filtered; dL/dC per pixel, then the state rewrite.
__global__ void __launch_bounds__(256) ssim_bwd_kernel(const float *__restrict__ img, const float *__restrict__ tgt,
                                                       int W, int H, SsimWindow win, const float *__restrict__ abc,
                                                       float lambda, float bg0, float bg1, float bg2,
                                                       float *__restrict__ state, float *__restrict__ grad_out) {
    __shared__ float ms[kSsimHH * kSsimHW * 3];
    __shared__ float hs[9][kSsimHH][kSsimTW];
    const int x0 = blockIdx.x * kSsimTW, y0 = blockIdx.y * kSsimTH;
    const int tid = threadIdx.x;
    const int64_t HW = (int64_t)W * H;
    for (int ch = 0; ch < 3; ++ch) {
        __syncthreads();
        // the three partials of this channel: a halo of a [H, W, 9] array restricted to 3 values
        for (int i = tid; i < kSsimHH * kSsimHW * 3; i += blockDim.x) {
            const int r = i / (kSsimHW * 3), e = i - r * (kSsimHW * 3);
            const int gy = y0 - kSsimR + r, gx = x0 - kSsimR + e / 3;
            ms[i] = (gx >= 0 && gx < W && gy >= 0 && gy < H) ? abc[((int64_t)gy * W + gx) * 9 + 3 * ch + e % 3]
                                                              : 0.f;
        }
        __syncthreads();
        for (int i = tid; i < kSsimHH * kSsimTW; i += blockDim.x) {
            const int r = i / kSsimTW, c = i - r * kSsimTW;
            const float *mr = ms + (r * kSsimHW + c) * 3;
            float fa = 0.f, fb = 0.f, fc = 0.f;
#pragma unroll
            for (int k = 0; k < kSsimK; ++k) {
                fa = fmaf(win.w[k], mr[3 * k + 0], fa);
                fb = fmaf(win.w[k], mr[3 * k + 1], fb);
                fc = fmaf(win.w[k], mr[3 * k + 2], fc);
            }
            hs[3 * ch + 0][r][c] = fa;
            hs[3 * ch + 1][r][c] = fb;
            hs[3 * ch + 2][r][c] = fc;
        }
    }
    __syncthreads();
    const int tx = tid & 31, ty = tid >> 5;
    const float inv_n = 1.f / (3.f * (float)HW);
    for (int rr = ty; rr < kSsimTH; rr += 8) {
        const int gx = x0 + tx, gy = y0 + rr;
        if (gx >= W || gy >= H) continue;
        const int64_t pix = (int64_t)gy * W + gx;
        float g[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            float fa = 0.f, fb = 0.f, fc = 0.f;
#pragma unroll
            for (int k = 0; k < kSsimK; ++k) {
                fa = fmaf(win.w[k], hs[3 * c + 0][rr + k][tx], fa);
                fb = fmaf(win.w[k], hs[3 * c + 1][rr + k][tx], fb);
                fc = fmaf(win.w[k], hs[3 * c + 2][rr + k][tx], fc);
            }
            const float x = img[3 * pix + c], y = tgt[3 * pix + c];
            const float dS = fa + 2.f * x * fb + y * fc;
            const float d = x - y;
            const float sg = d > 0.f ? 1.f : (d < 0.f ? -1.f : 0.f);
            g[c] = ((1.f - lambda) * sg - lambda * dS) * inv_n;
            if (grad_out) grad_out[3 * pix + c] = g[c];
        }
        // the forward left F (3), T, Q in the state planes; turn them into the backward state
        const float F0 = state[pix], F1 = state[HW + pix], F2 = state[2 * HW + pix];
        const float T = state[3 * HW + pix], Q = state[4 * HW + pix];
        const float Bq = Q > 0.f ? (1.f - T) / Q : 0.f;
        state[pix] = Bq * g[0];
        state[HW + pix] = Bq * g[1];
        state[2 * HW + pix] = Bq * g[2];
        state[3 * HW + pix] = T * (g[0] * (F0 - bg0) + g[1] * (F1 - bg1) + g[2] * (F2 - bg2));
        state[4 * HW + pix] = -Bq * (g[0] * F0 + g[1] * F1 + g[2] * F2);
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
