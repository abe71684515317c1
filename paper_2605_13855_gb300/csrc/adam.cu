// adam.cu -- sparse Adam over the active set (Sec. 5.1, "Implementation
// Details": the parameters are optimised with Adam; only the active set is
// optimised between active-set updates, Sec. 4.1).
//
// One launch, blockIdx.y = parameter group.  Within a group the threads run
// over the compact gradient rows (active order) element by element, so the
// compact gradients are read fully coalesced and each active splat's row of
// parameters and moments is a contiguous run of the group's width.
#include "common.cuh"
#include "launch.h"

namespace soit {

__global__ void __launch_bounds__(256) adam_kernel(const __grid_constant__ AdamArgs a) {
    const int k = blockIdx.y;
    const int w = a.width[k];
    const int64_t total = a.n_active * w;
    const float *__restrict__ g = a.g[k];
    float *__restrict__ p = a.p[k];
    float *__restrict__ m = a.m[k];
    float *__restrict__ v = a.v[k];
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = t / w;
        const int off = (int)(t - r * w);
        const int64_t e = a.active_rows ? t : (int64_t)a.idx[r] * w + off;  // parameter / moment element
        // colour SH: degree 0 (the first 3 floats of a row) has its own rate
        const float step = (k == 4 && off >= 3) ? a.step_size[5] : a.step_size[k == 5 ? 6 : k];
        const float gi = g[t];
        const float mi = fmaf(a.beta1, m[e], (1.f - a.beta1) * gi);
        const float vi = fmaf(a.beta2, v[e], (1.f - a.beta2) * gi * gi);
        m[e] = mi;
        v[e] = vi;
        p[e] -= step * mi / (sqrtf(vi) * a.inv_sqrt_bc2 + a.eps);
    }
    if (a.sigma_p && blockIdx.x == 0 && blockIdx.y == 0 && threadIdx.x == 0) {
        const float gi = *a.sigma_g;
        const float mi = fmaf(a.beta1, *a.sigma_m, (1.f - a.beta1) * gi);
        const float vi = fmaf(a.beta2, *a.sigma_v, (1.f - a.beta2) * gi * gi);
        *a.sigma_m = mi;
        *a.sigma_v = vi;
        *a.sigma_p -= a.step_size[7] * mi / (sqrtf(vi) * a.inv_sqrt_bc2 + a.eps);
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
    const int64_t most = a.n_active * 48;
    int64_t bx = (most + 255) / 256;
    if (bx < 1) bx = 1;
    if (bx > 152 * 16) bx = 152 * 16;  // grid-stride beyond 16 blocks per SM
    adam_kernel<<<dim3((unsigned)bx, 6), 256, 0, st>>>(a);
    return 0;
}

}  // namespace soit
