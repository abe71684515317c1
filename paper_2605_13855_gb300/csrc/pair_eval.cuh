// pair_eval.cuh -- the per-(splat, pixel) exponent of Eq. 5, shared by the
// forward and the backward rasters so that all of them take bit-identical
// contribution decisions.
//
// In tile-relative form: with the tile origin (ox, oy) = (16 tx + 0.5,
// 16 ty + 0.5), dx0 = ox - mu'x, dy0 = oy - mu'y, the pixel (kx, ky) of the
// tile has dy = dy0 + ky, u = dx0 + kx - r dy, and
//     e2 = B2 dy,  e1 = A2 u = (A2 dx0 - r A2 dy) + A2 kx,
//     -log2 alpha_raw = e1^2 + (e2^2 - log2 o).
// The row term nlrow = e2^2 - log2 o is one rounded FMA per row, so a pixel
// costs two: e1 = A2 kx + e10 and nlg = e1 e1 + nlrow (no negated operand).
// The pair contributes iff nlg <= log2 255 (alpha_raw >= 1/255) and then
// alpha_raw = 2^-nlg.  Every operation is explicitly rounded (no contraction
// differences between the kernels that inline it).
#pragma once
#include "common.cuh"

namespace soit {

// -log2 alpha_raw at or below this: the pair contributes (alpha_raw >= 1/255).
constexpr float kMaxNegLog2Alpha = kLog2_255;

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
    float dy;     // dy0 + ky
    float e10;    // e1 at kx = 0
    float nlrow;  // e2^2 - log2 o
};

__device__ __forceinline__ RowTerms row_terms(float A2dx0, float dy0, float rA2, float B2, float log2o, int ky) {
    RowTerms t;
    t.dy = __fadd_rn(dy0, (float)ky);
    const float e2 = __fmul_rn(B2, t.dy);
    t.nlrow = __fmaf_rn(e2, e2, -log2o);
    t.e10 = __fmaf_rn(-rA2, t.dy, A2dx0);
    return t;
}

__device__ __forceinline__ float col_e1(float A2, float e10, int kx) { return __fmaf_rn(A2, (float)kx, e10); }

// -log2 alpha_raw = e1^2 + nlrow (one rounding).
__device__ __forceinline__ float pair_nlg(float e1, float nlrow) { return __fmaf_rn(e1, e1, nlrow); }

// The same for two pixels per paired instruction; each component rounds like pair_nlg.
__device__ __forceinline__ float2 pair_nlg2(float2 e1, float2 nlrow) { return __ffma2_rn(e1, e1, nlrow); }

// Bound that every pixel of the tile stays under when the tile's four corner
// pixels do: the cutoff set is convex, and the margin (far above the rounding
// of nlg) keeps every pixel's rounded exponent inside the cut.
__device__ __forceinline__ float full_tile_lim(float log2o) {
    return kMaxNegLog2Alpha - fmaf(1e-3f, fabsf(log2o + kLog2_255), 1e-3f);
}

// The whole 16x16 tile lies inside the splat's cutoff ellipse.
__device__ __forceinline__ bool tile_inside(const SplatConsts &c, float A2, float B2, float log2o) {
    const float lim = full_tile_lim(log2o);
    bool in = true;
#pragma unroll
    for (int cyy = 0; cyy < 2; ++cyy) {
        const RowTerms rt = row_terms(c.A2dx0, c.dy0, c.rA2, B2, log2o, cyy * (kTile - 1));
#pragma unroll
        for (int cxx = 0; cxx < 2; ++cxx) in = in && pair_nlg(col_e1(A2, rt.e10, cxx * (kTile - 1)), rt.nlrow) <= lim;
    }
    return in;
}

// 2^x by the PTX approximate base-2 exponential (inputs here are in
// [-log2 255, 0]; relative error ~2^-22).  alpha_raw = fast_exp2(-nlg).
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

}  // namespace soit
