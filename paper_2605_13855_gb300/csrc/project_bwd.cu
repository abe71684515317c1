// project_bwd.cu -- chain rule from the screen-space gradients of each
// projected record (mu'x, mu'y, r, A2, B2, ln o, w, c) to the splat
// parameters: Eq. 6 (EWA projection), Eq. 2 (covariance from quaternion and
// scales), Eq. 4 (SH colour), Eq. 1 (OIT weight and sigma), Sec. 3.1
// (opacity = sigmoid(logit)).  One thread per active splat; the views of the
// batch are summed in registers and every gradient row is written once.  The
// block's SH coefficient rows (48 + 16 values a splat) pass through shared
// memory: the block copies them in, and its gradient rows out, with
// coalesced 16-byte accesses, and each thread reads and writes its own
// (padded) row there; per-thread global accesses to 192- and 64-byte rows
// would touch a different cache line in every lane of each warp access.
#include "common.cuh"
#include "launch.h"

namespace soit {

constexpr int kChainThreads = 128;
constexpr int kRowC4 = 13;  // float4 per staged colour row (12 + 1: consecutive rows land on different banks)
constexpr int kRowW4 = 5;   // float4 per staged weight row (4 + 1)

// Row r of the block (parameter row pi) into the staging rows, as FP32.
template <typename ShT>
__device__ __forceinline__ void stage_sh_rows(const SplatPtrs &sp, const int *list, int r0, int nb, float4 *shc,
                                              float4 *shw) {
    constexpr int kC16 = 48 * (int)sizeof(ShT) / 16, kW16 = 16 * (int)sizeof(ShT) / 16;  // 16-byte chunks a row
    constexpr int kPer = 16 / (int)sizeof(ShT);                                           // values a chunk
    for (int idx = threadIdx.x; idx < nb * (kC16 + kW16); idx += kChainThreads) {
        const int row = idx / (kC16 + kW16), part = idx - row * (kC16 + kW16);
        const int pi = sp.active_rows ? r0 + row : list[r0 + row];
        const bool colour = part < kC16;
        const int c = colour ? part : part - kC16;
        const ShT *src = reinterpret_cast<const ShT *>(colour ? sp.sh_color : sp.sh_weight) +
                         (int64_t)pi * (colour ? 48 : 16) + c * kPer;
        float *dst = reinterpret_cast<float *>(colour ? shc + row * kRowC4 : shw + row * kRowW4) + c * kPer;
        if (sizeof(ShT) == 4) {
            *reinterpret_cast<float4 *>(dst) = __ldg(reinterpret_cast<const float4 *>(src));
        } else {
            const uint4 raw = __ldg(reinterpret_cast<const uint4 *>(src));
            const uint32_t w[4] = {raw.x, raw.y, raw.z, raw.w};
#pragma unroll
            for (int k = 0; k < 4; ++k) {  // bf16 pair -> two floats (bf16 is the top half of an fp32)
                dst[2 * k] = __uint_as_float(w[k] << 16);
                dst[2 * k + 1] = __uint_as_float(w[k] & 0xffff0000u);
            }
        }
    }
}

// SH coefficients c0 .. c0 + 3 of the thread's staged rows (colour layout (r0 g0 b0 r1) (g1 b1 r2 g2) ...).
__device__ __forceinline__ void staged_sh_run(const float4 *hc, const float4 *hw, int c0, float h0[4], float h1[4],
                                              float h2[4], float hv[4]) {
    const float4 a = hc[3 * c0 / 4], b = hc[3 * c0 / 4 + 1], c = hc[3 * c0 / 4 + 2];
    h0[0] = a.x; h1[0] = a.y; h2[0] = a.z;
    h0[1] = a.w; h1[1] = b.x; h2[1] = b.y;
    h0[2] = b.z; h1[2] = b.w; h2[2] = c.x;
    h0[3] = c.y; h1[3] = c.z; h2[3] = c.w;
    const float4 w = hw[c0 / 4];
    hv[0] = w.x; hv[1] = w.y; hv[2] = w.z; hv[3] = w.w;
}

template <typename ShT>
__global__ void __launch_bounds__(kChainThreads, 3) project_bwd_kernel(const __grid_constant__ Batch b, SplatPtrs sp,
                                                          const int *__restrict__ list, int n,
                                                          const float4 *__restrict__ sgrad, GradPtrs out,
                                                          float *__restrict__ sig_part, unsigned *sig_count) {
    __shared__ float red[4];
    __shared__ int last_s;
    __shared__ float4 shc[kChainThreads * kRowC4], shw[kChainThreads * kRowW4];
    const int r0 = blockIdx.x * kChainThreads, nb = min(kChainThreads, n - r0);
    stage_sh_rows<ShT>(sp, list, r0, nb, shc, shw);
    __syncthreads();
    const int r = r0 + threadIdx.x;
    float4 *myc = shc + threadIdx.x * kRowC4, *myw = shw + threadIdx.x * kRowW4;
    float gsig_local = 0.f;
    if (r < n) {
        const int i = list[r];
        const int pi = sp.active_rows ? r : i;  // parameter row
        float mu[3], q[4], ls[3];
        for (int k = 0; k < 3; ++k) mu[k] = __ldg(sp.means + 3 * (int64_t)pi + k);
        const float4 q4 = __ldg(reinterpret_cast<const float4 *>(sp.quats) + pi);
        q[0] = q4.x; q[1] = q4.y; q[2] = q4.z; q[3] = q4.w;
        for (int k = 0; k < 3; ++k) ls[k] = __ldg(sp.log_scales + 3 * (int64_t)pi + k);
        const float ol = __ldg(sp.opacity_logits + pi);
        const float o = 1.f / (1.f + expf(-ol));
        // the staged rows and the parameters above are inputs of the step; the screen-space sums
        // below are the backward raster's output
        pdl_wait();
        pdl_allow_next();

        float g_mu[3] = {0.f, 0.f, 0.f}, g_q[4] = {0.f, 0.f, 0.f, 0.f}, g_ls[3] = {0.f, 0.f, 0.f}, g_ol = 0.f;
        float g_h[48], g_hw[16];
#pragma unroll
        for (int k = 0; k < 48; ++k) g_h[k] = 0.f;
#pragma unroll
        for (int k = 0; k < 16; ++k) g_hw[k] = 0.f;

        for (int v = 0; v < b.n_views; ++v) {
            const ViewDesc &vd = b.v[v];
            const int64_t qidx = (int64_t)v * n + r;
            const float4 G0 = sgrad[3 * qidx + 0], G1 = sgrad[3 * qidx + 1];
            const float2 G2 = *reinterpret_cast<const float2 *>(sgrad + 3 * qidx + 2);
            if (G0.x == 0.f && G0.y == 0.f && G0.z == 0.f && G0.w == 0.f && G1.x == 0.f && G1.y == 0.f &&
                G1.z == 0.f && G1.w == 0.f && G2.x == 0.f && G2.y == 0.f)
                continue;  // not binned in this view (culled or off-screen): no contribution
            SplatGeom g;
            if (!(o >= (1.f / 255.f)) || !splat_geometry(vd, mu, q, ls, g)) continue;
            const float gmx = G0.x, gmy = G0.y, gr = G0.z, gA2 = G0.w;
            const float gB2 = G1.x, glno = G1.y, gw = G1.z;
            const float gc[3] = {G1.w, G2.x, G2.y};
            const float z = g.tc[2], iz = 1.f / z;

            // (r, A2, B2) -> Sigma' entries (sxy the single off-diagonal value)
            const float A2 = sqrtf(kLog2e * g.syy / (2.f * g.det));
            const float B2 = sqrtf(kLog2e / (2.f * g.syy));
            const float isyy = 1.f / g.syy, idet = 1.f / g.det;
            const float g_sxx = gA2 * (-0.5f * A2 * g.syy * idet);
            const float g_syy = gA2 * (-0.5f * A2 * g.sxy * g.sxy * isyy * idet) - gB2 * 0.5f * B2 * isyy -
                                gr * g.sxy * isyy * isyy;
            const float g_sxy = gA2 * (A2 * g.sxy * idet) + gr * isyy;
            // sxx = |n0|^2 + 0.3, syy = |n1|^2 + 0.3, sxy = n0.n1
            float gn0[3], gn1[3];
            for (int k = 0; k < 3; ++k) {
                gn0[k] = 2.f * g_sxx * g.n0[k] + g_sxy * g.n1[k];
                gn1[k] = 2.f * g_syy * g.n1[k] + g_sxy * g.n0[k];
            }
            // n_k[b] = (J Qm)[k][b] s[b]
            const float j00 = vd.fx * iz, j02 = -vd.fx * g.tc[0] * iz * iz;
            const float j11 = vd.fy * iz, j12 = -vd.fy * g.tc[1] * iz * iz;
            float ga0[3], ga1[3];
            for (int k = 0; k < 3; ++k) {
                ga0[k] = gn0[k] * g.s[k];
                ga1[k] = gn1[k] * g.s[k];
                g_ls[k] += gn0[k] * g.n0[k] + gn1[k] * g.n1[k];  // d/dlog s = s d/ds, n = a s
            }
            // a0 = j00 Qm[0,:] + j02 Qm[2,:],  a1 = j11 Qm[1,:] + j12 Qm[2,:]
            float gj00 = 0.f, gj02 = 0.f, gj11 = 0.f, gj12 = 0.f;
            float gQm[9];
            for (int k = 0; k < 3; ++k) {
                gj00 += ga0[k] * g.Qm[0 * 3 + k];
                gj02 += ga0[k] * g.Qm[2 * 3 + k];
                gj11 += ga1[k] * g.Qm[1 * 3 + k];
                gj12 += ga1[k] * g.Qm[2 * 3 + k];
                gQm[0 * 3 + k] = j00 * ga0[k];
                gQm[1 * 3 + k] = j11 * ga1[k];
                gQm[2 * 3 + k] = j02 * ga0[k] + j12 * ga1[k];
            }
            // Qm = W Rq  ->  dL/dRq = W^T dL/dQm
            float gR[9];
            for (int a = 0; a < 3; ++a)
                for (int c = 0; c < 3; ++c)
                    gR[3 * a + c] = vd.R[0 * 3 + a] * gQm[0 * 3 + c] + vd.R[1 * 3 + a] * gQm[1 * 3 + c] +
                                    vd.R[2 * 3 + a] * gQm[2 * 3 + c];
            // J entries and mu' as functions of the camera-space centre t
            const float x = g.tc[0], y = g.tc[1];
            float gt0 = gj02 * (-vd.fx * iz * iz) + gmx * vd.fx * iz;
            float gt1 = gj12 * (-vd.fy * iz * iz) + gmy * vd.fy * iz;
            float gt2 = gj00 * (-vd.fx * iz * iz) + gj02 * (2.f * vd.fx * x * iz * iz * iz) +
                        gj11 * (-vd.fy * iz * iz) + gj12 * (2.f * vd.fy * y * iz * iz * iz) -
                        (gmx * vd.fx * x + gmy * vd.fy * y) * iz * iz;
            // SH basis at the view direction
            const float idl = 1.f / g.dlen;
            const float nx = g.d[0] * idl, ny = g.d[1] * idl, nz = g.d[2] * idl;
            float Y[16];
            sh_basis16(nx, ny, nz, Y);
            float craw[3] = {0.5f, 0.5f, 0.5f}, vraw = 0.5f;
#pragma unroll
            for (int q4 = 0; q4 < 4; ++q4) {  // coefficients 4 q4 .. 4 q4 + 3, vector loads
                float h0[4], h1[4], h2[4], hv[4];
                staged_sh_run(myc, myw, 4 * q4, h0, h1, h2, hv);
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const int k = 4 * q4 + j;
                    craw[0] = fmaf(Y[k], h0[j], craw[0]);
                    craw[1] = fmaf(Y[k], h1[j], craw[1]);
                    craw[2] = fmaf(Y[k], h2[j], craw[2]);
                    vraw = fmaf(Y[k], hv[j], vraw);
                }
            }
            // Eq. 1: w = max(0, 1 - z/sigma) max(0, vraw)
            const float zterm = 1.f - z / sp.sigma;
            float gv = 0.f;
            if (zterm > 0.f) {
                const float vv = fmaxf(vraw, 0.f);
                gv = gw * zterm;
                gt2 -= gw * vv / sp.sigma;
                gsig_local += gw * vv * z / (sp.sigma * sp.sigma);
            }
            // Eq. 4 colour / weight SH coefficients and the direction gradient
            float coef[16];
            const float m0 = craw[0] > 0.f ? gc[0] : 0.f, m1 = craw[1] > 0.f ? gc[1] : 0.f,
                        m2 = craw[2] > 0.f ? gc[2] : 0.f, mv = vraw > 0.f ? gv : 0.f;
#pragma unroll
            for (int q4 = 0; q4 < 4; ++q4) {
                float h0[4], h1[4], h2[4], hv[4];
                staged_sh_run(myc, myw, 4 * q4, h0, h1, h2, hv);
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const int k = 4 * q4 + j;
                    g_h[3 * k + 0] = fmaf(m0, Y[k], g_h[3 * k + 0]);
                    g_h[3 * k + 1] = fmaf(m1, Y[k], g_h[3 * k + 1]);
                    g_h[3 * k + 2] = fmaf(m2, Y[k], g_h[3 * k + 2]);
                    g_hw[k] = fmaf(mv, Y[k], g_hw[k]);
                    coef[k] = m0 * h0[j] + m1 * h1[j] + m2 * h2[j] + mv * hv[j];
                }
            }
            float gdir[3];
            sh_grad16(nx, ny, nz, coef, gdir);
            const float ndot = nx * gdir[0] + ny * gdir[1] + nz * gdir[2];
            // t = W mu + t_w; dir = (mu - campos)/|mu - campos|
            g_mu[0] += vd.R[0] * gt0 + vd.R[3] * gt1 + vd.R[6] * gt2 + (gdir[0] - nx * ndot) * idl;
            g_mu[1] += vd.R[1] * gt0 + vd.R[4] * gt1 + vd.R[7] * gt2 + (gdir[1] - ny * ndot) * idl;
            g_mu[2] += vd.R[2] * gt0 + vd.R[5] * gt1 + vd.R[8] * gt2 + (gdir[2] - nz * ndot) * idl;
            // opacity: d ln(sigmoid(l)) / dl = 1 - o
            g_ol += glno * (1.f - o);
            // R(q^): derivative of each entry in (a, b, c, d) = (w, x, y, z)
            const float qa = g.qn[0], qb = g.qn[1], qc = g.qn[2], qd = g.qn[3];
            float gqa = 2.f * (-qd * gR[1] + qc * gR[2] + qd * gR[3] - qb * gR[5] - qc * gR[6] + qb * gR[7]);
            float gqb = 2.f * (qc * gR[1] + qd * gR[2] + qc * gR[3] - 2.f * qb * gR[4] - qa * gR[5] + qd * gR[6] +
                               qa * gR[7] - 2.f * qb * gR[8]);
            float gqc = 2.f * (-2.f * qc * gR[0] + qb * gR[1] + qa * gR[2] + qb * gR[3] + qd * gR[5] - qa * gR[6] +
                               qd * gR[7] - 2.f * qc * gR[8]);
            float gqd = 2.f * (-2.f * qd * gR[0] - qa * gR[1] + qb * gR[2] + qa * gR[3] - 2.f * qd * gR[4] +
                               qc * gR[5] + qb * gR[6] + qc * gR[7]);
            const float qdot = qa * gqa + qb * gqb + qc * gqc + qd * gqd;
            const float iq = 1.f / g.qlen;
            g_q[0] += (gqa - qa * qdot) * iq;
            g_q[1] += (gqb - qb * qdot) * iq;
            g_q[2] += (gqc - qc * qdot) * iq;
            g_q[3] += (gqd - qd * qdot) * iq;
        }
        const int64_t row = out.rows_by_splat ? (int64_t)i : (int64_t)r;
        float4 *oq = reinterpret_cast<float4 *>(out.quats) + row;
        if (out.accumulate) {  // add to the caller's running sums (several backward calls)
            for (int k = 0; k < 3; ++k) g_mu[k] += out.means[3 * row + k];
            const float4 pq = *oq;
            g_q[0] += pq.x; g_q[1] += pq.y; g_q[2] += pq.z; g_q[3] += pq.w;
            for (int k = 0; k < 3; ++k) g_ls[k] += out.log_scales[3 * row + k];
            g_ol += out.opacity_logits[row];
        }
        for (int k = 0; k < 3; ++k) out.means[3 * row + k] = g_mu[k];
        *oq = make_float4(g_q[0], g_q[1], g_q[2], g_q[3]);
        for (int k = 0; k < 3; ++k) out.log_scales[3 * row + k] = g_ls[k];
        out.opacity_logits[row] = g_ol;
        // the SH gradient rows into the thread's own staging rows (its parameter reads are done)
#pragma unroll
        for (int k = 0; k < 12; ++k) myc[k] = make_float4(g_h[4 * k], g_h[4 * k + 1], g_h[4 * k + 2], g_h[4 * k + 3]);
#pragma unroll
        for (int k = 0; k < 4; ++k) myw[k] = make_float4(g_hw[4 * k], g_hw[4 * k + 1], g_hw[4 * k + 2], g_hw[4 * k + 3]);
    }
    __syncthreads();
    // the block's SH gradient rows out, coalesced (added to the running sums when accumulating)
    for (int idx = threadIdx.x; idx < nb * 16; idx += kChainThreads) {
        const int row = idx >> 4, part = idx & 15;
        const int64_t orow = out.rows_by_splat ? (int64_t)list[r0 + row] : (int64_t)(r0 + row);
        float4 *dst = part < 12 ? reinterpret_cast<float4 *>(out.sh_color + 48 * orow) + part
                                : reinterpret_cast<float4 *>(out.sh_weight + 16 * orow) + (part - 12);
        float4 v = part < 12 ? shc[row * kRowC4 + part] : shw[row * kRowW4 + part - 12];
        if (out.accumulate) {
            const float4 o4 = *dst;
            v.x += o4.x; v.y += o4.y; v.z += o4.z; v.w += o4.w;
        }
        *dst = v;
    }
    // dL/dsigma: the block's sum to sig_part, then the last block to finish sums the partials in
    // block order (no float atomics on one address) and resets the counter for the next launch
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) gsig_local += __shfl_xor_sync(0xffffffffu, gsig_local, off);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = gsig_local;
    __syncthreads();
    if (threadIdx.x == 0) {
        sig_part[blockIdx.x] = red[0] + red[1] + red[2] + red[3];
        __threadfence();
        last_s = atomicAdd(sig_count, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!last_s) return;
    __threadfence();
    float sum = 0.f;
    for (int k = threadIdx.x; k < (int)gridDim.x; k += kChainThreads) sum += __ldcg(sig_part + k);
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, off);
    __syncthreads();  // red[] is read above by thread 0 only; reuse it
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = sum;
    __syncthreads();
    if (threadIdx.x == 0) {
        const float total = red[0] + red[1] + red[2] + red[3];
        *out.sigma = out.accumulate ? *out.sigma + total : total;
        *sig_count = 0u;
    }
}

int project_bwd_blocks(int n) { return (n + kChainThreads - 1) / kChainThreads; }

int launch_project_bwd(const Batch &b, const SplatPtrs &sp, bool bf16, const int *list, int n, const float4 *sgrad,
                       GradPtrs out, float *sig_part, unsigned *sig_count, bool pdl, cudaStream_t st) {
    if (n == 0) return 0;
    const int grid = project_bwd_blocks(n);
    if (bf16)
        launch_kernel(project_bwd_kernel<__nv_bfloat16>, dim3(grid), dim3(kChainThreads), st, pdl, b, sp, list, n,
                      sgrad, out, sig_part, sig_count);
    else
        launch_kernel(project_bwd_kernel<float>, dim3(grid), dim3(kChainThreads), st, pdl, b, sp, list, n, sgrad,
                      out, sig_part, sig_count);
    return 0;
}

}  // namespace soit
