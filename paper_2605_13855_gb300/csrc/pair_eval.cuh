// pair_eval.cuh -- the per-(splat, pixel) exponent of Eq. 5, shared by the
// forward and the backward rasters so that all of them take bit-identical
// contribution decisions.
//
// In tile-relative form: with the tile origin (ox, oy) = (16 tx + 0.5,
// 16 ty + 0.5), dx0 = ox - mu'x, dy0 = oy - mu'y, the pixel (kx, ky) of the
// tile has dy = dy0 + ky, u = dx0 + kx - r dy, and
//     e2 = B2 dy,  e1 = A2 u = (A2 dx0 - r A2 dy) + A2 kx,
//     log2 alpha_raw = (log2 o - e2^2) - e1^2.
// The row term lrow = log2 o - e2^2 is rounded once per row, so a pixel
// costs two fused multiply-adds: e1 = A2 kx + e10 and lg = lrow - e1 e1.
// The pair contributes iff lg >= -log2 255 (alpha_raw >= 1/255).  Every
// operation is explicitly rounded (no contraction differences between the
// kernels that inline it).
#pragma once
#include "common.cuh"

namespace soit {

// log2 alpha_raw at or above this: the pair contributes (alpha_raw >= 1/255).
constexpr float kMinLog2Alpha = -kLog2_255;

// Per-splat constants of the evaluation, computed identically wherever used:
// A2dx0 = A2 (ox - mu'x), dy0 = oy - mu'y, rA2 = r A2.
struct SplatConsts {
    float A2dx0, dy0, rA2;
};

__device__ __forceinline__ SplatConsts splat_consts(float ox, float oy, float mx, float my, float rr, float A2) {
    SplatConsts c;
    c.A2dx0 = __fmul_rn(A2, __fsub_rn(ox, mx));
    c.dy0 = __fsub_rn(oy, my);
    c.rA2 = __fmul_rn(rr, A2);
    return c;
}

struct RowTerms {
    float dy;    // dy0 + ky
    float e10;   // e1 at kx = 0
    float lrow;  // log2 o - e2^2
};

__device__ __forceinline__ RowTerms row_terms(float A2dx0, float dy0, float rA2, float B2, float log2o, int ky) {
    RowTerms t;
    t.dy = __fadd_rn(dy0, (float)ky);
    const float e2 = __fmul_rn(B2, t.dy);
    t.lrow = __fsub_rn(log2o, __fmul_rn(e2, e2));
    t.e10 = __fmaf_rn(-rA2, t.dy, A2dx0);
    return t;
}

__device__ __forceinline__ float col_e1(float A2, float e10, int kx) { return __fmaf_rn(A2, (float)kx, e10); }

// log2 alpha_raw = lrow - e1^2 (one rounding).
__device__ __forceinline__ float pair_lg(float e1, float lrow) { return __fmaf_rn(-e1, e1, lrow); }

// The same for two pixels per paired instruction; each component rounds like pair_lg.
__device__ __forceinline__ float2 pair_lg2(float2 e1, float2 lrow) {
    return __ffma2_rn(make_float2(-e1.x, -e1.y), e1, lrow);
}

// Bound below which every pixel of the tile contributes when the tile's four
// corner pixels reach it: the cutoff set is convex, and the margin (far above
// the rounding of lg) keeps every pixel's rounded exponent above the cut.
__device__ __forceinline__ float full_tile_lim(float log2o) {
    return kMinLog2Alpha + fmaf(1e-3f, fabsf(log2o - kMinLog2Alpha), 1e-3f);
}

// The whole 16x16 tile lies inside the splat's cutoff ellipse.
__device__ __forceinline__ bool tile_inside(const SplatConsts &c, float A2, float B2, float log2o) {
    const float lim = full_tile_lim(log2o);
    bool in = true;
#pragma unroll
    for (int cyy = 0; cyy < 2; ++cyy) {
        const RowTerms rt = row_terms(c.A2dx0, c.dy0, c.rA2, B2, log2o, cyy * (kTile - 1));
#pragma unroll
        for (int cxx = 0; cxx < 2; ++cxx) in = in && pair_lg(col_e1(A2, rt.e10, cxx * (kTile - 1)), rt.lrow) >= lim;
    }
    return in;
}

// 2^x by the PTX approximate base-2 exponential (inputs here are in
// [-log2 255, 0]; relative error ~2^-22).
__device__ __forceinline__ float fast_exp2(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// 1/x by the PTX approximate reciprocal (x in [0.01, 1] here).
__device__ __forceinline__ float fast_rcp(float x) {
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// Square root by the PTX approximate instruction (deterministic for a given input).
__device__ __forceinline__ float fast_sqrt(float x) {
    float y;
    asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// Columns [x0, x0 + 2 n) of one tile row, x0 even, that hold every pixel of the
// row whose exponent reaches the cut: |e1| <= R with R^2 = lrow + log2 255,
// i.e. kx in [(-R - e10) / A2, (R - e10) / A2].  R^2 is widened by 1e-5 and the
// columns by 0.02 px (both far above the rounding of lg, e1 and the
// approximate square root and reciprocal), so the span is a superset of the
// pixels the exact test accepts; the caller still tests each pixel.  n = 0:
// no pixel of the row can contribute.
__device__ __forceinline__ void row_span(float invA2, float e10, float lrow, int &x0, int &n) {
    const float R2 = __fadd_rn(lrow, kLog2_255 + 1e-5f);
    x0 = 0;
    n = 0;
    if (!(R2 > 0.f)) return;
    const float R = fast_sqrt(R2);
    const float xl = __fmul_rn(__fsub_rn(-R, e10), invA2), xr = __fmul_rn(__fsub_rn(R, e10), invA2);
    const int lo = f2i_clamped(ceilf(xl - 0.02f), 0, kTile);
    const int hi = f2i_clamped(floorf(xr + 0.02f), -1, kTile - 1);
    if (lo > hi) return;
    x0 = lo & ~1;
    n = ((hi - x0) >> 1) + 1;
}

}  // namespace soit
