// raster_bwd_pixel.cu -- per-pixel parallel backward raster, the baseline of
// the backward ablation (Sec. 5.3, Tab. 2: the 3DGS per-pixel backward
// against per-splat backwards).  Same gradients as raster_bwd.cu (Eq. 10
// chained to the screen-space record), organised the other way round:
// a thread owns a pixel, a block a 16 x 16 tile, and all threads walk the
// tile's splats together (staged in shared memory 256 at a time).  Each
// contributing pair yields the splat's ten screen-space sums for that pixel
//   (da e1, da e1 dy, da e1^2, da dy, da dy^2, da, a D, a B g_r, a B g_g, a B g_b)
// (notation of raster_bwd.cu), which reach the splat's accumulator either
//   kWarpReduce = false: one set of atomics per contributing pair (the 3DGS
//     scheme: every pixel adds into every splat it touches), or
//   kWarpReduce = true: summed over the warp's 32 pixels with shuffles first,
//     one set of atomics per (warp, splat).
// The exponent and the contribution test are the shared, explicitly rounded
// ones, so the pairs are exactly those of the forward.
#include "common.cuh"
#include "launch.h"
#include "pair_eval.cuh"

namespace soit {

constexpr int kPixBatch = 256;

template <bool kWarpReduce>
__global__ void __launch_bounds__(kTilePix) raster_bwd_pixel_kernel(const __grid_constant__ Batch b,
                                                                    const float4 *__restrict__ rec,
                                                                    const int *__restrict__ offsets,
                                                                    const uint32_t *__restrict__ pairs, int64_t cap,
                                                                    uint32_t nrec, float4 *__restrict__ sgrad) {
    // staged per splat: s0 = (A2 dx0, dy0, r A2, A2), s1 = (B2, 0, log2 o, w), s2 = (c_r, c_g, c_b, r)
    __shared__ float4 s0[kPixBatch], s1[kPixBatch], s2[kPixBatch];
    __shared__ uint32_t sq[kPixBatch];

    if (bin_failed(b)) return;  // the binning scan gave up: offsets and tile order are incomplete
    const int gt = block_tile(b);
    const int v = find_view(b, gt);
    const ViewDesc &vd = b.v[v];
    const int lt = gt - vd.tile_base;
    const int ty = lt / vd.tiles_x, tx = lt - ty * vd.tiles_x;
    const int tid = threadIdx.x, lane = tid & 31;
    const int kx = tid & (kTile - 1), ky = tid >> 4;
    const float ox = (float)(tx * kTile) + 0.5f, oy = (float)(ty * kTile) + 0.5f;

    // this pixel's state: B g (3), A, -B g.F (zero outside the image: contributes nothing)
    float Bg0 = 0.f, Bg1 = 0.f, Bg2 = 0.f, Ast = 0.f, nBgF = 0.f;
    {
        const int x = tx * kTile + kx, y = ty * kTile + ky;
        if (x < vd.W && y < vd.H) {
            const int64_t HW = (int64_t)vd.W * vd.H, pix = (int64_t)y * vd.W + x;
            const float *st = vd.state;
            Bg0 = st[pix];
            Bg1 = st[HW + pix];
            Bg2 = st[2 * HW + pix];
            Ast = st[3 * HW + pix];
            nBgF = st[4 * HW + pix];
        }
    }
    const int start = offsets[gt];
    const int end = (int)min((int64_t)offsets[gt + 1], cap);
    for (int base = start; base < end; base += kPixBatch) {
        const int n = min(kPixBatch, end - base);
        __syncthreads();
        if (tid < n) {
            const uint32_t q = pairs[base + tid];
            float4 t0 = make_float4(0.f, 0.f, 0.f, 0.f), t1 = make_float4(0.f, 0.f, -INFINITY, 0.f), t2 = t0;
            if (q < nrec) {
                const float4 a0 = rec[3 * (int64_t)q + 0];
                const float4 a1 = rec[3 * (int64_t)q + 1];
                const float4 a2 = rec[3 * (int64_t)q + 2];
                const SplatConsts c = splat_consts(ox, oy, a0.x, a0.y, a0.z, a0.w);
                t0 = make_float4(c.A2dx0, c.dy0, c.rA2, a0.w);
                t1 = make_float4(a1.x, 0.f, a1.y, a1.z);
                t2 = make_float4(a2.x, a2.y, a2.z, a0.z);
            }
            s0[tid] = t0;
            s1[tid] = t1;
            s2[tid] = t2;
            sq[tid] = q;
        }
        __syncthreads();
        for (int j = 0; j < n; ++j) {
            const float4 a0 = s0[j], a1 = s1[j];
            const RowTerms rt = row_terms(a0.x, a0.y, a0.z, a1.x, a1.z, ky);
            const float e1 = col_e1(a0.w, rt.e10, kx);
            const float nlg = pair_nlg(e1, rt.nlrow);
            const bool in = nlg <= kMaxNegLog2Alpha;
            if (!__any_sync(0xffffffffu, in)) continue;
            float v10[10];
#pragma unroll
            for (int k = 0; k < 10; ++k) v10[k] = 0.f;
            if (in) {
                const float4 a2 = s2[j];
                const float ar = fast_exp2(-nlg);
                const float a = fminf(ar, kAlphaMax);
                const float am = ar > kAlphaMax ? 0.f : a;
                const float D = fmaf(Bg0, a2.x, fmaf(Bg1, a2.y, fmaf(Bg2, a2.z, nBgF)));
                const float dLda = fmaf(Ast, fast_rcp(1.f - a), a1.w * D);
                const float da = dLda * am;
                const float de = da * e1;
                v10[0] = de;
                v10[1] = de * rt.dy;
                v10[2] = de * e1;
                v10[3] = da * rt.dy;
                v10[4] = da * rt.dy * rt.dy;
                v10[5] = da;
                v10[6] = a * D;
                v10[7] = a * Bg0;
                v10[8] = a * Bg1;
                v10[9] = a * Bg2;
            }
            bool emit = in;
            if (kWarpReduce) {
#pragma unroll
                for (int k = 0; k < 10; ++k)
#pragma unroll
                    for (int off = 16; off > 0; off >>= 1) v10[k] += __shfl_xor_sync(0xffffffffu, v10[k], off);
                emit = lane == 0;
            }
            if (emit) {
                const uint32_t q = sq[j];
                const float A2 = a0.w, B2 = a1.x, w = a1.w, rr = s2[j].w;
                const float K = -2.f * kLn2;
                float4 *out = sgrad + 3 * (int64_t)q;
                atomicAdd(out + 0, make_float4(-K * A2 * v10[0], K * (A2 * rr * v10[0] - B2 * B2 * v10[3]),
                                               -K * A2 * v10[1], K * v10[2] / A2));
                atomicAdd(out + 1, make_float4(K * B2 * v10[4], v10[5], v10[6], w * v10[7]));
                atomicAdd(reinterpret_cast<float2 *>(out + 2), make_float2(w * v10[8], w * v10[9]));
            }
        }
    }
}

int launch_raster_bwd_pixel(const Batch &b, bool warp_reduce, const float4 *rec, const int *offsets,
                            const uint32_t *pairs, int64_t cap, float4 *sgrad, cudaStream_t st) {
    if (b.total_tiles == 0) return 0;
    const uint32_t nrec = (uint32_t)((int64_t)b.n_views * b.n_list);
    if (warp_reduce)
        raster_bwd_pixel_kernel<true><<<b.total_tiles, kTilePix, 0, st>>>(b, rec, offsets, pairs, cap, nrec, sgrad);
    else
        raster_bwd_pixel_kernel<false><<<b.total_tiles, kTilePix, 0, st>>>(b, rec, offsets, pairs, cap, nrec, sgrad);
    return 0;
}

}  // namespace soit
