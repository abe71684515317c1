// pair_eval.cuh -- the per-(splat, pixel) exponent of Eq. 5, shared by the
// forward and the backward raster so that both take bit-identical
// contribution decisions.
//
// In tile-relative form: with the tile origin (ox, oy) = (16 tx + 0.5,
// 16 ty + 0.5), dx0 = ox - mu'x, dy0 = oy - mu'y, the pixel (kx, ky) of the
// tile has dy = dy0 + ky, u = dx0 + kx - r dy, and
//     e2 = B2 dy,  e1 = A2 u = (A2 dx0 - r A2 dy) + A2 kx,
//     log2 alpha_raw = log2 o - (e1^2 + e2^2).
// Every operation is explicitly rounded (no contraction differences between
// the kernels that inline it).
#pragma once
#include "common.cuh"

namespace soit {

// Per-splat constants of the evaluation, computed identically wherever used:
// A2dx0 = A2 (ox - mu'x), rA2 = r A2, thr = log2 o + log2 255 (the pair
// contributes iff s = e1^2 + e2^2 <= thr, i.e. alpha_raw >= 1/255).
struct SplatConsts {
    float A2dx0, dy0, rA2, thr;
};

__device__ __forceinline__ SplatConsts splat_consts(float ox, float oy, float mx, float my, float rr, float A2,
                                                    float log2o) {
    SplatConsts c;
    c.A2dx0 = __fmul_rn(A2, __fsub_rn(ox, mx));
    c.dy0 = __fsub_rn(oy, my);
    c.rA2 = __fmul_rn(rr, A2);
    c.thr = __fadd_rn(log2o, kLog2_255);
    return c;
}

struct RowTerms {
    float dy, e2sq, e10;  // e10 = e1 at kx = 0
};

__device__ __forceinline__ RowTerms row_terms(float A2dx0, float dy0, float rA2, float B2, int ky) {
    RowTerms t;
    t.dy = __fadd_rn(dy0, (float)ky);
    const float e2 = __fmul_rn(B2, t.dy);
    t.e2sq = __fmul_rn(e2, e2);
    t.e10 = __fmaf_rn(-rA2, t.dy, A2dx0);
    return t;
}

__device__ __forceinline__ float col_e1(float A2, float e10, int kx) { return __fmaf_rn(A2, (float)kx, e10); }

// s = e1^2 + e2^2; contributes iff s <= thr; log2 alpha_raw = log2 o - s.
__device__ __forceinline__ float quad_s(float e1, float e2sq) { return __fmaf_rn(e1, e1, e2sq); }

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

}  // namespace soit
