// adam.cu -- sparse Adam over the active set (Sec. 5.1, "Implementation
// Details": the parameters are optimised with Adam; only the active set is
// optimised between active-set updates, Sec. 4.1).
//
// One launch, blockIdx.y = parameter group.  Within a group the threads run
// over the compact gradient rows (active order), so the compact gradients are
// read fully coalesced and each active splat's row of parameters and moments
// is a contiguous run of the group's width, moved in 16-byte accesses where
// the width allows (adam_group).
#include "common.cuh"
#include "launch.h"

namespace soit {

// One Adam update of element values (g, p, m, v) -> (p, m, v) with step size `step`.
__device__ __forceinline__ void adam_one(const AdamArgs &a, float step, float gi, float &p, float &m, float &v) {
    m = fmaf(a.beta1, m, (1.f - a.beta1) * gi);
    v = fmaf(a.beta2, v, (1.f - a.beta2) * gi * gi);
    p -= step * m / (sqrtf(v) * a.inv_sqrt_bc2 + a.eps);
}

// Step size of element `off` of a row of group k: the colour SH's degree-0 coefficients (the first
// 3 floats of a row) have their own rate.
__device__ __forceinline__ float adam_step(const AdamArgs &a, int k, int off) {
    return (k == 4 && off >= 3) ? a.step_size[5] : a.step_size[k == 5 ? 6 : k];
}

__device__ __forceinline__ void adam_vec(const AdamArgs &a, int k, int off0, float4 g, float4 *pp, float4 *mp,
                                         float4 *vp) {
    float4 p = *pp, m = *mp, v = *vp;
    adam_one(a, adam_step(a, k, off0 + 0), g.x, p.x, m.x, v.x);
    adam_one(a, adam_step(a, k, off0 + 1), g.y, p.y, m.y, v.y);
    adam_one(a, adam_step(a, k, off0 + 2), g.z, p.z, m.z, v.z);
    adam_one(a, adam_step(a, k, off0 + 3), g.w, p.w, m.w, v.w);
    *pp = p;
    *mp = m;
    *vp = v;
}

// Group k of row width W.  Stage layout (active_rows): the four arrays are dense [n_active, W] in the
// same order, so the group is one flat run, updated four floats per 16-byte access (the rows of
// width 48 start every 192 bytes, so a chunk never straddles two rows) and the last total % 4
// elements one by one.  Rows by splat: a row of width 4, 16 or 48 is gathered through the index
// list in 16-byte chunks, rows of width 1 or 3 element by element.  `vec`: the arrays are 16-byte
// aligned (else every group takes the element path).
template <int W>
__device__ __forceinline__ void adam_group(const AdamArgs &a, int k, bool vec) {
    const float *__restrict__ g = a.g[k];
    float *__restrict__ p = a.p[k];
    float *__restrict__ m = a.m[k];
    float *__restrict__ v = a.v[k];
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t t0 = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t total = a.n_active * W;
    if (a.active_rows && vec) {
        const int64_t n4 = total / 4;
        for (int64_t c = t0; c < n4; c += stride)
            adam_vec(a, k, (int)((4 * c) % W), reinterpret_cast<const float4 *>(g)[c],
                     reinterpret_cast<float4 *>(p) + c, reinterpret_cast<float4 *>(m) + c,
                     reinterpret_cast<float4 *>(v) + c);
        for (int64_t t = 4 * n4 + t0; t < total; t += stride)
            adam_one(a, adam_step(a, k, (int)(t % W)), g[t], p[t], m[t], v[t]);
    } else if (W % 4 == 0 && vec) {
        constexpr int C = W % 4 == 0 ? W / 4 : 1;  // chunks a row (the branch is taken for W % 4 == 0 only)
        const int64_t nc = a.n_active * C;
        for (int64_t c = t0; c < nc; c += stride) {
            const int64_t r = c / C;
            const int j = (int)(c - r * C);
            const int64_t e4 = (a.active_rows ? r : (int64_t)a.idx[r]) * C + j;
            adam_vec(a, k, 4 * j, reinterpret_cast<const float4 *>(g)[c], reinterpret_cast<float4 *>(p) + e4,
                     reinterpret_cast<float4 *>(m) + e4, reinterpret_cast<float4 *>(v) + e4);
        }
    } else {
        for (int64_t t = t0; t < total; t += stride) {
            const int64_t r = t / W;
            const int off = (int)(t - r * W);
            const int64_t e = a.active_rows ? t : (int64_t)a.idx[r] * W + off;
            adam_one(a, adam_step(a, k, off), g[t], p[e], m[e], v[e]);
        }
    }
}

// One launch, blockIdx.y = parameter group (means, quats, log_scales, opacity, sh_color, sh_weight).
__global__ void __launch_bounds__(256) adam_kernel(const __grid_constant__ AdamArgs a, int vec_mask) {
    const int k = blockIdx.y;
    const bool vec = (vec_mask >> k) & 1;
    switch (k) {
        case 0: adam_group<3>(a, k, vec); break;
        case 1: adam_group<4>(a, k, vec); break;
        case 2: adam_group<3>(a, k, vec); break;
        case 3: adam_group<1>(a, k, vec); break;
        case 4: adam_group<48>(a, k, vec); break;
        default: adam_group<16>(a, k, vec); break;
    }
    if (a.sigma_p && blockIdx.x == 0 && blockIdx.y == 0 && threadIdx.x == 0) {
        float pp = *a.sigma_p, mm = *a.sigma_m, vv = *a.sigma_v;
        adam_one(a, a.step_size[7], *a.sigma_g, pp, mm, vv);
        *a.sigma_m = mm;
        *a.sigma_v = vv;
        *a.sigma_p = pp;
    }
}

// Gather (to_active) or scatter of the active rows of one group's arrays: active[t] <->
// full[idx[r] w + off], t = r w + off, elements of type T.
template <typename T>
__global__ void __launch_bounds__(256) rows_copy_kernel(const int *__restrict__ idx, int64_t n_active, int w,
                                                        const T *__restrict__ src, T *__restrict__ dst,
                                                        bool to_active) {
    const int64_t total = n_active * w;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = t / w;
        const int64_t e = (int64_t)idx[r] * w + (t - r * w);
        if (to_active)
            dst[t] = src[e];
        else
            dst[e] = src[t];
    }
}

int launch_rows_copy(const int *idx, int64_t n_active, int w, const void *src, void *dst, int elem_bytes,
                     bool to_active, cudaStream_t st) {
    const int64_t total = n_active * w;
    if (total == 0) return 0;
    int64_t bx = (total + 255) / 256;
    if (bx > 152 * 16) bx = 152 * 16;
    if (elem_bytes == 2)
        rows_copy_kernel<uint16_t><<<(unsigned)bx, 256, 0, st>>>(idx, n_active, w, (const uint16_t *)src,
                                                                 (uint16_t *)dst, to_active);
    else
        rows_copy_kernel<float><<<(unsigned)bx, 256, 0, st>>>(idx, n_active, w, (const float *)src, (float *)dst,
                                                              to_active);
    return 0;
}

int launch_adam(const AdamArgs &a, cudaStream_t st) {
    if (a.n_active == 0 && !a.sigma_p) return 0;
    const int width[6] = {3, 4, 3, 1, 48, 16};
    int vec_mask = 0;
    for (int k = 0; k < 6; ++k) {
        const bool aligned = ((uintptr_t)a.g[k] | (uintptr_t)a.p[k] | (uintptr_t)a.m[k] | (uintptr_t)a.v[k]) % 16 == 0;
        if (aligned && (a.active_rows || width[k] % 4 == 0)) vec_mask |= 1 << k;
    }
    const int64_t most = (a.n_active * 48 + 3) / 4;  // chunks of the widest group
    int64_t bx = (most + 255) / 256;
    if (bx < 1) bx = 1;
    if (bx > 152 * 16) bx = 152 * 16;  // grid-stride beyond 16 blocks per SM
    adam_kernel<<<dim3((unsigned)bx, 6), 256, 0, st>>>(a, vec_mask);
    return 0;
}

}  // namespace soit
