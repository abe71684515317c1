// active_update.cu -- the periodic active-set update (Sec. 4.1, Eq. 8;
// Alg. 1, the IsActiveUpdateIteration branch).
//
// The update renders the full set on a farthest-point subsample of the
// training views, sums the gradients over those views (the renderer's
// backward with accumulate = 1 and rows indexed by splat), and keeps a splat
// active when the gradient of at least one of its attribute groups has a
// norm above that group's threshold.  This file holds the two pieces that
// are new to that loop: the view subsampling (host) and the activeness test
// (one pass over the N x 75 gradient rows).
#include <cmath>
#include <cstdint>
#include <vector>

#include "common.cuh"
#include "sparseoit.h"

namespace soit {

constexpr int kActBlock = 128;     // splats per block

// floats per splat of each attribute group: mu, q, log s, opacity logit, colour SH, weight SH
__host__ __device__ constexpr int group_width(int k) {
    return k == 0 ? 3 : k == 1 ? 4 : k == 2 ? 3 : k == 3 ? 1 : k == 4 ? 48 : 16;
}

// Loads the block's contiguous chunk [first*w, (first+cnt)*w) of a row-major
// [n, w] array into shared memory (coalesced; 16-byte vectors when aligned).
__device__ __forceinline__ void load_rows(const float *__restrict__ src, int w, int64_t first, int cnt,
                                          float *__restrict__ buf) {
    const int64_t f0 = first * w;
    const int nf = cnt * w;
    const float *p = src + f0;
    if ((reinterpret_cast<uintptr_t>(p) & 15) == 0) {
        const int nv = nf >> 2;
        const float4 *p4 = reinterpret_cast<const float4 *>(p);
        for (int k = threadIdx.x; k < nv; k += blockDim.x) reinterpret_cast<float4 *>(buf)[k] = __ldg(p4 + k);
        for (int k = (nv << 2) + threadIdx.x; k < nf; k += blockDim.x) buf[k] = __ldg(p + k);
    } else {
        for (int k = threadIdx.x; k < nf; k += blockDim.x) buf[k] = __ldg(p + k);
    }
}

struct ActArgs {
    const float *g[6];
    float eps[6];
    int64_t n;
    uint8_t *mask;
    float *norms;
};

__global__ void __launch_bounds__(kActBlock) activeness_kernel(const __grid_constant__ ActArgs a) {
    __shared__ __align__(16) float buf[kActBlock * 48];
    const int64_t first = (int64_t)blockIdx.x * kActBlock;
    const int cnt = (int)min((int64_t)kActBlock, a.n - first);
    const int t = threadIdx.x;
    float nrm[6];
    bool active = false;
#pragma unroll
    for (int k = 0; k < 6; ++k) {
        const int w = group_width(k);
        __syncthreads();
        load_rows(a.g[k], w, first, cnt, buf);
        __syncthreads();
        float ss = 0.f;
        if (t < cnt)
            for (int j = 0; j < w; ++j) ss = fmaf(buf[t * w + j], buf[t * w + j], ss);
        nrm[k] = sqrtf(ss);
        active |= nrm[k] > a.eps[k];
    }
    if (t < cnt) {
        const int64_t i = first + t;
        a.mask[i] = active ? 1 : 0;
        if (a.norms)
#pragma unroll
            for (int k = 0; k < 6; ++k) a.norms[6 * i + k] = nrm[k];
    }
}

}  // namespace soit

extern "C" {

int sparseoit_fps_views(const sparseoit_camera *cams, int32_t n, int32_t s, int32_t first, int32_t *out) {
    if (!cams || !out || n < 1 || s < 1 || s > n || first < 0 || first >= n) return SPARSEOIT_ERR_INVALID_ARG;
    // camera centres c = -R^T t (R row-major, world to camera), in double
    std::vector<double> c(3 * (size_t)n);
    for (int j = 0; j < n; ++j) {
        const float *R = cams[j].R, *t = cams[j].t;
        for (int k = 0; k < 3; ++k) {
            const double p0 = (double)R[k] * t[0], p1 = (double)R[3 + k] * t[1], p2 = (double)R[6 + k] * t[2];
            c[3 * j + k] = -((p0 + p1) + p2);
        }
    }
    // d[j] = squared distance from view j to the nearest chosen view
    std::vector<double> d(n, INFINITY);
    int cur = first;
    for (int k = 0; k < s; ++k) {
        out[k] = cur;
        const double cx = c[3 * cur], cy = c[3 * cur + 1], cz = c[3 * cur + 2];
        int best = -1;
        double bd = -1.0;
        for (int j = 0; j < n; ++j) {
            const double dx = c[3 * j] - cx, dy = c[3 * j + 1] - cy, dz = c[3 * j + 2] - cz;
            const double sx = dx * dx, sy = dy * dy, sz = dz * dz;
            const double dd = (sx + sy) + sz;
            if (dd < d[j]) d[j] = dd;
            if (d[j] > bd) {
                bd = d[j];
                best = j;
            }
        }
        cur = best;
    }
    return SPARSEOIT_OK;
}

int sparseoit_activeness(const sparseoit_grads *g, int64_t n, const float *eps, uint8_t *d_mask, float *d_norms,
                         void *stream) {
    if (!g || !eps || !d_mask || n < 0) return SPARSEOIT_ERR_INVALID_ARG;
    if (!g->means || !g->quats || !g->log_scales || !g->opacity_logits || !g->sh_color || !g->sh_weight)
        return SPARSEOIT_ERR_INVALID_ARG;
    if (n == 0) return SPARSEOIT_OK;
    soit::ActArgs a;
    a.g[0] = g->means;
    a.g[1] = g->quats;
    a.g[2] = g->log_scales;
    a.g[3] = g->opacity_logits;
    a.g[4] = g->sh_color;
    a.g[5] = g->sh_weight;
    for (int k = 0; k < 6; ++k) a.eps[k] = eps[k];
    a.n = n;
    a.mask = d_mask;
    a.norms = d_norms;
    const int64_t blocks = (n + soit::kActBlock - 1) / soit::kActBlock;
    if (blocks > 0x7fffffffll) return SPARSEOIT_ERR_INVALID_ARG;
    soit::activeness_kernel<<<(unsigned)blocks, soit::kActBlock, 0, (cudaStream_t)stream>>>(a);
    return cudaGetLastError() == cudaSuccess ? SPARSEOIT_OK : SPARSEOIT_ERR_CUDA;
}

}  // extern "C"
