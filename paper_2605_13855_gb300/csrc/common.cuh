// common.cuh -- device-side definitions shared by the kernels of libsparseoit.
//
// Data layout in HBM (one batch = the views of one forward / commit call):
//   * projected record of list entry r in batch view v: index q = v * n_list + r,
//       rec[3q+0] = (mu'x, mu'y, r, A2)        quadratic form, see below
//       rec[3q+1] = (B2, log2 o, w, yh)        yh = y half-extent of the cutoff ellipse
//       rec[3q+2] = (c_r, c_g, c_b, sign)      sign = +1 / -1 (frozen-sum update)
//     ext[q] = (tau2', y half-extent, 1 / A2, dy of the x extreme)
//   * tile bins: one tile id space for all views of the batch (view v owns
//     [tile_base, tile_base + tiles_x * tiles_y)); offsets[t] .. offsets[t+1]
//     index the u32 pair arena that holds record indices q (no depth key).
//   * per-pixel planes (H*W floats each): frozen sums (P_r, P_g, P_b, Q, log T)
//     and the backward pixel state (B g_r, B g_g, B g_b, A, -B g.F).
//
// The per-pair exponent is evaluated in a factored form of Eq. 5 that has no
// cancellation for thin ellipses:  with Sigma' = [[sxx, sxy], [sxy, syy]],
//     1/2 d^T Sigma'^-1 d = syy/(2 det) (dx - (sxy/syy) dy)^2 + dy^2/(2 syy),
// so with L = log2(e), r = sxy/syy, A2 = sqrt(L syy / (2 det)),
// B2 = sqrt(L / (2 syy)):
//     log2 alpha_raw = log2 o - (A2 (dx - r dy))^2 - (B2 dy)^2.
#pragma once
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace soit {

constexpr int kTile = 16;                       // tile edge in pixels (App. A: 16x16 tiles)
constexpr int kTilePix = kTile * kTile;         // 256 pixels = 8 warps (Sec. 4.2)
constexpr int kMaxViews = 32;
constexpr float kNearZ = 0.2f;                  // near-plane cull (3DGS convention)
constexpr float kDilation = 0.3f;               // low-pass dilation of Sigma' (3DGS convention)
constexpr float kAlphaMax = 0.99f;              // opacity clamp (3DGS convention)
// About log2(0.989): a splat with log2 o at or below it never reaches the clamp.
// Its raw alpha is 2^(log2 o - s) with s >= 0, at most 2^-0.015957 = 0.98900
// before the approximate exp2 errs by a few ulp (1e-5 relative would still
// stay below 0.99), so the rasters skip min(., 0.99) for it with identical
// results.
constexpr float kNoClampLog2 = -0.015957f;
constexpr float kLog2e = 1.4426950408889634f;
constexpr float kLn2 = 0.6931471805599453f;
constexpr float kLog2_255 = 7.9943534368588578f;  // log2(255); alpha_raw >= 1/255 <=> log2 alpha_raw >= -this

constexpr unsigned kStatusCapacity = 1u;
constexpr unsigned kStatusTimeout = 2u;

struct ViewDesc {
    float R[9], t[3];             // world -> camera
    float fx, fy, cx, cy;
    float campos[3];              // camera centre -R^T t
    int W, H, tiles_x, tiles_y;
    int tile_base;                // first batch tile id of this view
    int pad_;
    float *image;                 // [H, W, 3] output image (forward)
    const float *target;          // [H, W, 3] L1 target (fused loss) or null
    float *frozen;                // 5 planes: frozen sums of this view
    float *state;                 // 5 planes: pixel state (or F, T, Q before prep)
    const float *grad_image;      // [H, W, 3] dL/dC (unfused backward) or null
};

struct Batch {
    int n_views;
    int total_tiles;
    int n_list;                   // list entries (records) per view
    int pad_;
    const int *tile_order;        // raster block -> global tile (heaviest first); null = identity
    const unsigned *status;       // device status word (kStatusTimeout: the binning scan gave up)
    ViewDesc v[kMaxViews];
};

// Programmatic dependent launch (sm_90 and later).  The kernels of a step
// are launched so that a kernel's blocks may become resident while the
// kernel before it on the stream drains.  A kernel calls pdl_wait() before
// it reads anything that kernel writes (griddepcontrol.wait returns once the
// previous grid has completed and its memory operations are visible), and
// pdl_allow_next() after that wait, so that the next kernel's early part
// only ever runs once every kernel before this one has completed.  Launched
// without the attribute, both are no-ops.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_allow_next() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

// The tile scan of this batch's binning gave up (a bounded wait ran out): its
// offsets and tile order are incomplete, so the kernels after it do nothing.
// (Read through the read-only cache: no kernel after the scan writes the
// word, and the one line is then fetched once per SM instead of once per warp.)
__device__ __forceinline__ bool bin_failed(const Batch &b) {
    return b.status && (__ldg(b.status) & kStatusTimeout);
}

// The per-tile pair counters of the projection sit 64 bytes apart (a stride
// of 16 ints): neighbouring tiles are often all heavy, and adjacent counters
// send all their atomics to one L2 slice (measured at 1M splats / 5 %: the
// busiest slice's atomic unit 64 % busy against 8 % on average with dense
// counters; the projection 35 us dense, 24 us at 32 bytes, 19 us at 64 and at
// 128).  The scatter's cursors stay dense (their position-returning atomics
// measured faster that way).
constexpr int kTileCounterStride = 16;

// Binning scan (project.cu): partitions of kScanItems tiles, one block of
// kScanThreads threads each; per-batch scratch (zeroed before every scan).
constexpr int kScanThreads = 256, kScanPer = 4, kScanItems = kScanThreads * kScanPer;
constexpr int kLoadClasses = 128;  // raster tile-order classes (four per octave of pair count)
struct ScanScratch {
    unsigned long long *state;    // [partitions] posted aggregate / inclusive prefix
    int *ticket;                  // next partition number
    int *class_hist;              // [kLoadClasses] tiles per load class
    int *class_cursor;            // [kLoadClasses] placement counters of the tile order
};
inline int scan_partitions(int total) { return total > 0 ? (total + kScanItems - 1) / kScanItems : 1; }
// Bytes of the scratch for `tiles` tiles, and its layout in one allocation.
inline size_t scan_scratch_bytes(int64_t tiles) {
    return (size_t)scan_partitions((int)tiles) * 8 + (2 + 2 * kLoadClasses) * sizeof(int);
}
inline ScanScratch scan_scratch_at(void *p, int64_t tiles) {
    ScanScratch s;
    s.state = reinterpret_cast<unsigned long long *>(p);
    s.ticket = reinterpret_cast<int *>(s.state + scan_partitions((int)tiles));
    s.class_hist = s.ticket + 2;
    s.class_cursor = s.class_hist + kLoadClasses;
    return s;
}

// Global tile a raster block works on: blocks are handed out heaviest tile
// first, so that the long tiles start early instead of forming the tail.
__device__ __forceinline__ int block_tile(const Batch &b) {
    return b.tile_order ? __ldg(b.tile_order + blockIdx.x) : (int)blockIdx.x;
}

struct SplatPtrs {
    const float *means, *quats, *log_scales, *opacity_logits;
    const void *sh_color, *sh_weight;
    float sigma;
    float bg[3];
    int active_rows;  // 1: row r of every array is the r-th active splat (else row i is splat i)
};

__device__ __forceinline__ int find_view(const Batch &b, int gt) {
    int v = 0;
    while (v + 1 < b.n_views && gt >= b.v[v + 1].tile_base) ++v;
    return v;
}

// Clamp a float to [lo, hi] before converting (NaN -> lo).
__device__ __forceinline__ int f2i_clamped(float f, int lo, int hi) {
    if (!(f >= (float)lo)) return lo;
    if (f >= (float)hi) return hi;
    return (int)f;
}

template <typename T>
__device__ __forceinline__ float ldf(const T *p, int64_t i);
template <>
__device__ __forceinline__ float ldf<float>(const float *p, int64_t i) { return __ldg(p + i); }
template <>
__device__ __forceinline__ float ldf<__nv_bfloat16>(const __nv_bfloat16 *p, int64_t i) {
    return __bfloat162float(p[i]);
}

// Real orthonormal spherical harmonics of degree <= 3 at the unit vector
// (x, y, z), without the Condon-Shortley phase, index k = l^2 + l + m
// (Eq. 4).  Each constant is sqrt((2l+1)/(4 pi) (l-|m|)!/(l+|m|)!) times the
// factors of the Cartesian polynomial (and sqrt 2 for m != 0), written out.
namespace shc {
constexpr float C0 = 0.28209479177387814f;   // sqrt(1/(4 pi))
constexpr float C1 = 0.48860251190291992f;   // sqrt(3/(4 pi))
constexpr float C2a = 1.0925484305920792f;   // sqrt(15/(4 pi))       xy, yz, xz
constexpr float C2b = 0.31539156525252005f;  // sqrt(5/(16 pi))       3z^2 - 1
constexpr float C2c = 0.54627421529603959f;  // sqrt(15/(16 pi))      x^2 - y^2
constexpr float C3a = 0.59004358992664352f;  // sqrt(35/(32 pi))      3x^2 y - y^3, x^3 - 3 x y^2
constexpr float C3b = 2.8906114426405538f;   // sqrt(105/(4 pi))      xyz
constexpr float C3c = 0.45704579946446577f;  // sqrt(21/(32 pi))      y(5z^2-1), x(5z^2-1)
constexpr float C3d = 0.37317633259011540f;  // sqrt(7/(16 pi))       z(5z^2 - 3)
constexpr float C3e = 1.4453057213202771f;   // sqrt(105/(16 pi))     z(x^2 - y^2)
}  // namespace shc

__device__ __forceinline__ void sh_basis16(float x, float y, float z, float Y[16]) {
    using namespace shc;
    const float xx = x * x, yy = y * y, zz = z * z;
    Y[0] = C0;
    Y[1] = C1 * y;
    Y[2] = C1 * z;
    Y[3] = C1 * x;
    Y[4] = C2a * x * y;
    Y[5] = C2a * y * z;
    Y[6] = C2b * (3.f * zz - 1.f);
    Y[7] = C2a * x * z;
    Y[8] = C2c * (xx - yy);
    Y[9] = C3a * y * (3.f * xx - yy);
    Y[10] = C3b * x * y * z;
    Y[11] = C3c * y * (5.f * zz - 1.f);
    Y[12] = C3d * z * (5.f * zz - 3.f);
    Y[13] = C3c * x * (5.f * zz - 1.f);
    Y[14] = C3e * z * (xx - yy);
    Y[15] = C3a * x * (xx - 3.f * yy);
}

// Gradient, in (x, y, z) as free variables, of f = sum_k a_k Y_k.
__device__ __forceinline__ void sh_grad16(float x, float y, float z, const float a[16], float g[3]) {
    using namespace shc;
    const float xx = x * x, yy = y * y, zz = z * z;
    float gx = 0.f, gy = 0.f, gz = 0.f;
    gy += a[1] * C1;
    gz += a[2] * C1;
    gx += a[3] * C1;
    gx += a[4] * C2a * y;              gy += a[4] * C2a * x;
    gy += a[5] * C2a * z;              gz += a[5] * C2a * y;
    gz += a[6] * 6.f * C2b * z;
    gx += a[7] * C2a * z;              gz += a[7] * C2a * x;
    gx += a[8] * 2.f * C2c * x;        gy -= a[8] * 2.f * C2c * y;
    gx += a[9] * 6.f * C3a * x * y;    gy += a[9] * 3.f * C3a * (xx - yy);
    gx += a[10] * C3b * y * z;         gy += a[10] * C3b * x * z;   gz += a[10] * C3b * x * y;
    gy += a[11] * C3c * (5.f * zz - 1.f);  gz += a[11] * 10.f * C3c * y * z;
    gz += a[12] * C3d * (15.f * zz - 3.f);
    gx += a[13] * C3c * (5.f * zz - 1.f);  gz += a[13] * 10.f * C3c * x * z;
    gx += a[14] * 2.f * C3e * x * z;   gy -= a[14] * 2.f * C3e * y * z;  gz += a[14] * C3e * (xx - yy);
    gx += a[15] * 3.f * C3a * (xx - yy);   gy -= a[15] * 6.f * C3a * x * y;
    g[0] = gx; g[1] = gy; g[2] = gz;
}

// Cooperative SH evaluation by a group of G lanes (G = 1, 2, 4 or 16): lane
// k of the group holds the J = 16 / G consecutive coefficients J k, ...,
// J k + J - 1 (one contiguous run of the splat's row, loaded as vectors);
// yk[j] is the basis value of coefficient J k + j, picked without dynamic
// register indexing.
template <int G>
__device__ __forceinline__ void sh_basis_group(float x, float y, float z, int k, float yk[16 / G]) {
    constexpr int J = 16 / G;
    float Y[16];
    sh_basis16(x, y, z, Y);
#pragma unroll
    for (int j = 0; j < J; ++j) {
        float v = Y[j];
#pragma unroll
        for (int m = 1; m < G; ++m) v = (k == m) ? Y[J * m + j] : v;
        yk[j] = v;
    }
}

// The J consecutive colour (3 per coefficient) and weight coefficients from
// coefficient c0 of one splat's rows hc [16, 3] and hw [16]: 16-byte vector
// loads for FP32 with J = 4 (rows are 192 and 64 bytes, so every run is
// 16-byte aligned), scalar loads otherwise.
template <typename T, int J>
__device__ __forceinline__ void load_sh_run(const T *hc, const T *hw, int c0, float h0[J], float h1[J], float h2[J],
                                            float hv[J]) {
#pragma unroll
    for (int j = 0; j < J; ++j) {
        h0[j] = ldf(hc, 3 * (c0 + j) + 0);
        h1[j] = ldf(hc, 3 * (c0 + j) + 1);
        h2[j] = ldf(hc, 3 * (c0 + j) + 2);
        hv[j] = ldf(hw, c0 + j);
    }
}
template <>
__device__ __forceinline__ void load_sh_run<float, 4>(const float *hc, const float *hw, int c0, float h0[4],
                                                      float h1[4], float h2[4], float hv[4]) {
    const float4 *c4 = reinterpret_cast<const float4 *>(hc + 3 * c0);
    const float4 a = __ldg(c4), b = __ldg(c4 + 1), c = __ldg(c4 + 2);
    // (r0 g0 b0 r1) (g1 b1 r2 g2) (b2 r3 g3 b3)
    h0[0] = a.x; h1[0] = a.y; h2[0] = a.z;
    h0[1] = a.w; h1[1] = b.x; h2[1] = b.y;
    h0[2] = b.z; h1[2] = b.w; h2[2] = c.x;
    h0[3] = c.y; h1[3] = c.z; h2[3] = c.w;
    const float4 w = __ldg(reinterpret_cast<const float4 *>(hw + c0));
    hv[0] = w.x; hv[1] = w.y; hv[2] = w.z; hv[3] = w.w;
}

// Mask of the G lanes of this lane's group (groups are aligned in the warp).
template <int G>
__device__ __forceinline__ unsigned group_mask() {
    return (G == 32) ? 0xffffffffu : (((1u << G) - 1u) << (threadIdx.x & 31 & ~(G - 1)));
}

// Sum of v over the G lanes of this lane's group (result in every lane); all
// G lanes must call it together.
template <int G>
__device__ __forceinline__ float group_sum(float v, unsigned mask) {
#pragma unroll
    for (int off = G / 2; off > 0; off >>= 1) v += __shfl_xor_sync(mask, v, off);
    return v;
}

// Rotation of the unit quaternion (w, x, y, z), row-major.
__device__ __forceinline__ void quat_rot(float a, float b, float c, float d, float R[9]) {
    R[0] = 1.f - 2.f * (c * c + d * d); R[1] = 2.f * (b * c - a * d);       R[2] = 2.f * (b * d + a * c);
    R[3] = 2.f * (b * c + a * d);       R[4] = 1.f - 2.f * (b * b + d * d); R[5] = 2.f * (c * d - a * b);
    R[6] = 2.f * (b * d - a * c);       R[7] = 2.f * (c * d + a * b);       R[8] = 1.f - 2.f * (b * b + c * c);
}

// Geometry of one splat in one view (Eq. 2 and Eq. 6), shared by the forward
// projection and the backward chain so that both see identical values.
struct SplatGeom {
    float tc[3];          // camera-space centre
    float s[3];           // axis scales
    float Rq[9];          // rotation of the unit quaternion
    float qn[4], qlen;    // unit quaternion, |q|
    float Qm[9];          // W Rq
    float n0[3], n1[3];   // rows of N = J W Rq S
    float sxx, sxy, syy, det;
    float d[3], dlen;     // mu - camera centre, its length
};

__device__ __forceinline__ bool splat_geometry(const ViewDesc &vd, const float mu[3], const float q[4],
                                               const float ls[3], SplatGeom &g) {
    for (int r = 0; r < 3; ++r)
        g.tc[r] = fmaf(vd.R[3 * r + 0], mu[0], fmaf(vd.R[3 * r + 1], mu[1], fmaf(vd.R[3 * r + 2], mu[2], vd.t[r])));
    const float z = g.tc[2];
    if (!(z > kNearZ)) return false;
    g.qlen = sqrtf(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
    const float iq = 1.f / g.qlen;
    for (int k = 0; k < 4; ++k) g.qn[k] = q[k] * iq;
    quat_rot(g.qn[0], g.qn[1], g.qn[2], g.qn[3], g.Rq);
    for (int k = 0; k < 3; ++k) g.s[k] = expf(ls[k]);
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b)
            g.Qm[3 * a + b] = fmaf(vd.R[3 * a + 0], g.Rq[0 * 3 + b],
                                   fmaf(vd.R[3 * a + 1], g.Rq[1 * 3 + b], vd.R[3 * a + 2] * g.Rq[2 * 3 + b]));
    // rows of J: j0 = (fx/z, 0, -fx x/z^2), j1 = (0, fy/z, -fy y/z^2)
    const float iz = 1.f / z;
    const float j00 = vd.fx * iz, j02 = -vd.fx * g.tc[0] * iz * iz;
    const float j11 = vd.fy * iz, j12 = -vd.fy * g.tc[1] * iz * iz;
    for (int b = 0; b < 3; ++b) {
        g.n0[b] = fmaf(j00, g.Qm[0 * 3 + b], j02 * g.Qm[2 * 3 + b]) * g.s[b];
        g.n1[b] = fmaf(j11, g.Qm[1 * 3 + b], j12 * g.Qm[2 * 3 + b]) * g.s[b];
    }
    const float nn0 = g.n0[0] * g.n0[0] + g.n0[1] * g.n0[1] + g.n0[2] * g.n0[2];
    const float nn1 = g.n1[0] * g.n1[0] + g.n1[1] * g.n1[1] + g.n1[2] * g.n1[2];
    g.sxx = nn0 + kDilation;
    g.syy = nn1 + kDilation;
    g.sxy = g.n0[0] * g.n1[0] + g.n0[1] * g.n1[1] + g.n0[2] * g.n1[2];
    // det(N N^T) = |n0 x n1|^2 (Cauchy-Binet).  n0 x n1 = fx fy s0 s1 s2 / z^3
    // * (Rq^T (mu - campos)) / s (componentwise), a sum of squares with no
    // cancellation; det(N N^T + 0.3 I) = det(N N^T) + 0.3 tr(N N^T) + 0.09.
    for (int k = 0; k < 3; ++k) g.d[k] = mu[k] - vd.campos[k];
    g.dlen = sqrtf(g.d[0] * g.d[0] + g.d[1] * g.d[1] + g.d[2] * g.d[2]);
    float cb = 0.f;
    for (int k = 0; k < 3; ++k) {
        float lk = (g.Rq[0 * 3 + k] * g.d[0] + g.Rq[1 * 3 + k] * g.d[1] + g.Rq[2 * 3 + k] * g.d[2]) / g.s[k];
        cb = fmaf(lk, lk, cb);
    }
    const float kz = vd.fx * vd.fy * g.s[0] * g.s[1] * g.s[2] * iz * iz * iz;
    const float detNN = kz * kz * cb;
    g.det = detNN + kDilation * (nn0 + nn1) + kDilation * kDilation;
    return true;
}

}  // namespace soit
