/*
 * sparseoit_oracle.c -- plain FP64 CPU oracle of the SparseOIT renderer
 * (weighted-sum order-independent-transparency Gaussian splatting, forward
 * and backward, with the active / frozen split of the active-set method).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the reference the CUDA path is
 * checked against.  Only the test-suite, the smoke check and the CPU
 * baseline of the benchmark load it; the product library never does, and
 * the two share no code, header, table or constant.
 *
 * Everything is double precision and written as the plain definition:
 *
 *   Eq. 2   3D Gaussian, Sigma = R S S^T R^T (R from the unit quaternion,
 *           S = diag(exp(log_scale))).
 *   Eq. 6   EWA projection Sigma' = J W Sigma W^T J^T, J the Jacobian of the
 *           pinhole map at the camera-space centre, plus a 0.3 px^2 low-pass
 *           dilation on the diagonal (3DGS convention, Sec. 5.1 "other
 *           settings follow 3DGS").
 *   Eq. 5   alpha = o * exp(-1/2 d^T Sigma'^-1 d) (the exponential that the
 *           printed equation lost), clamped to 0.99 and dropped below 1/255.
 *   Eq. 4   colour c = max(0, Y(dir) . h + 0.5), dir the unit vector from the
 *           camera centre to the mean, Y the real orthonormal SH of degree 3.
 *   Eq. 1   OIT weight w = max(0, 1 - d/sigma) v, d = camera-space depth,
 *           v = max(0, Y(dir) . h_w + 0.5) a single-channel degree-3 SH
 *           (Sec. 5.1 states v is single channel).
 *   Eq. 7/9 C = T c0 + (1 - T) F, F = P/Q, P = sum c a w, Q = sum a w,
 *           T = prod (1 - a); F := 0 when Q = 0.
 *   Eq. 10  dC/dc_i, dC/dalpha_i, dC/dw_i, chained by hand through Eq. 5,
 *           6, 2, 4 and 1 to every splat parameter.
 *   Sec. 4.1 the frozen complement's contribution is kept as the per-pixel
 *           sums (P, Q, log T) so that sums(A) + sums(complement) are the
 *           sums of the whole set.
 *
 * Pixel (x, y) has its centre at (x + 0.5, y + 0.5).  Sums are accumulated
 * per pixel in ascending splat index, so the binned and the brute-force
 * renders below give bit-identical results.
 *
 * Parity of this oracle with the paper's own renderer is unpinned: the
 * paper prints no worked example.  Its arithmetic is pinned instead by the
 * CPU tests (brute force, closed forms, invariants, SciPy's spherical
 * harmonics, central finite differences).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_NEAR_Z     0.2          /* near-plane cull: t_z <= 0.2 is dropped   */
#define OR_DILATION   0.3          /* added to the diagonal of Sigma'          */
#define OR_ALPHA_MIN  (1.0 / 255.0)
#define OR_ALPHA_MAX  0.99
#define OR_NPARAM     75           /* 3 + 4 + 3 + 1 + 48 + 16                  */
#define OR_BAND       16           /* rows per bin of the binned render        */

/* ---------------------------------------------------------------- SH --- */

/* (2m-1)!! with (-1)!! = 1 */
static double double_factorial_odd(int m) {
    double r = 1.0;
    for (int k = 2 * m - 1; k > 1; k -= 2) r *= (double)k;
    return r;
}

static double factorial(int n) {
    double r = 1.0;
    for (int k = 2; k <= n; ++k) r *= (double)k;
    return r;
}

/* Pbar[l][m](z) = d^m P_l(z) / dz^m for 0 <= m <= l <= 3 (the associated
 * Legendre function without Condon-Shortley phase and without the
 * (1-z^2)^(m/2) factor), by the standard three-term recursion in l. */
static void legendre_bar(double z, double Pb[4][5]) {
    for (int l = 0; l < 4; ++l)
        for (int m = 0; m < 5; ++m) Pb[l][m] = 0.0;
    for (int m = 0; m <= 3; ++m) {
        Pb[m][m] = double_factorial_odd(m);
        if (m + 1 <= 3) Pb[m + 1][m] = (2.0 * m + 1.0) * z * Pb[m][m];
        for (int l = m + 2; l <= 3; ++l)
            Pb[l][m] = ((2.0 * l - 1.0) * z * Pb[l - 1][m] - (l + m - 1.0) * Pb[l - 2][m]) / (double)(l - m);
    }
}

/* Real orthonormal SH of degree <= 3, index k = l^2 + l + m:
 *   Y_l0      = K_l0 Pbar_l^0(z)
 *   Y_lm      = sqrt2 K_lm Pbar_l^m(z) Re((x + i y)^m)      (m > 0)
 *   Y_l,-m    = sqrt2 K_lm Pbar_l^m(z) Im((x + i y)^m)      (m > 0)
 * with K_lm = sqrt((2l+1)/(4 pi) (l-m)!/(l+m)!).  On the unit sphere this is
 * the usual real basis without the Condon-Shortley phase.  Y is evaluated as
 * a polynomial in (x, y, z); dY (optional, [16][3]) is its gradient in
 * (x, y, z) treated as free variables.  d/dz Pbar_l^m = Pbar_l^{m+1},
 * d/dx (x+iy)^m = m (x+iy)^(m-1), d/dy (x+iy)^m = i m (x+iy)^(m-1). */
void oracle_sh_basis(const double n[3], double Y[16], double *dY) {
    const double x = n[0], y = n[1], z = n[2];
    double Pb[4][5];
    legendre_bar(z, Pb);
    double Re[5], Im[5];
    Re[0] = 1.0; Im[0] = 0.0;
    for (int m = 1; m <= 4; ++m) {
        Re[m] = x * Re[m - 1] - y * Im[m - 1];
        Im[m] = x * Im[m - 1] + y * Re[m - 1];
    }
    for (int l = 0; l <= 3; ++l) {
        for (int m = 0; m <= l; ++m) {
            double K = sqrt((2.0 * l + 1.0) / (4.0 * M_PI) * factorial(l - m) / factorial(l + m));
            if (m == 0) {
                int k = l * l + l;
                Y[k] = K * Pb[l][0];
                if (dY) {
                    dY[3 * k + 0] = 0.0;
                    dY[3 * k + 1] = 0.0;
                    dY[3 * k + 2] = K * (l >= 1 ? Pb[l][1] : 0.0);
                }
            } else {
                double c = sqrt(2.0) * K;
                int kp = l * l + l + m, km = l * l + l - m;
                double P = Pb[l][m], dP = (m + 1 <= l) ? Pb[l][m + 1] : 0.0;
                Y[kp] = c * P * Re[m];
                Y[km] = c * P * Im[m];
                if (dY) {
                    /* d Re_m/dx = m Re_{m-1}, d Re_m/dy = -m Im_{m-1}
                     * d Im_m/dx = m Im_{m-1}, d Im_m/dy =  m Re_{m-1} */
                    dY[3 * kp + 0] = c * P * m * Re[m - 1];
                    dY[3 * kp + 1] = -c * P * m * Im[m - 1];
                    dY[3 * kp + 2] = c * dP * Re[m];
                    dY[3 * km + 0] = c * P * m * Im[m - 1];
                    dY[3 * km + 1] = c * P * m * Re[m - 1];
                    dY[3 * km + 2] = c * dP * Im[m];
                }
            }
        }
    }
}

/* ------------------------------------------------------------ camera --- */

/* cam[16]: R (world->camera rotation, row-major, OpenCV axes x right,
 * y down, z forward), t, fx, fy, cx, cy.  A world point X maps to the
 * camera-space point R X + t and to the pixel (fx x/z + cx, fy y/z + cy). */
typedef struct {
    double R[9], t[3], fx, fy, cx, cy, pos[3];
} ocam;

static void load_camera(const double *cam, ocam *c) {
    memcpy(c->R, cam, 9 * sizeof(double));
    memcpy(c->t, cam + 9, 3 * sizeof(double));
    c->fx = cam[12]; c->fy = cam[13]; c->cx = cam[14]; c->cy = cam[15];
    /* camera centre = -R^T t */
    for (int i = 0; i < 3; ++i)
        c->pos[i] = -(c->R[0 * 3 + i] * c->t[0] + c->R[1 * 3 + i] * c->t[1] + c->R[2 * 3 + i] * c->t[2]);
}

/* -------------------------------------------------------- projection --- */

typedef struct {
    int valid;              /* 0: culled by the near plane or o < 1/255      */
    double t[3];            /* camera-space centre                           */
    double m2[2];           /* pixel-space centre mu'                        */
    double Sig[9];          /* 3D covariance (Eq. 2)                         */
    double Rq[9], s[3];     /* rotation of the unit quaternion, scales       */
    double qn[4], qlen;     /* unit quaternion (w, x, y, z) and |q|          */
    double J[6], Tm[6];     /* EWA Jacobian J (2x3) and J W (2x3)            */
    double cov[3];          /* Sigma' (xx, xy, yy), dilation included        */
    double con[3];          /* Sigma'^-1 (xx, xy, yy)                        */
    double o;               /* opacity                                       */
    double c_raw[3], c[3];  /* colour before / after max(0, .)               */
    double v_raw, v;        /* weight SH before / after max(0, .)            */
    double zterm, w;        /* 1 - t_z/sigma and the OIT weight (Eq. 1)      */
    double n[3], dlen;      /* unit view direction, |mu - camera centre|     */
    double Y[16];           /* SH basis at n                                 */
    int x0, x1, y0, y1;     /* conservative pixel bbox (inclusive), clipped  */
} oproj;

static void quat_to_rot(const double q[4], double R[9]) {
    const double a = q[0], b = q[1], c = q[2], d = q[3];
    R[0] = 1.0 - 2.0 * (c * c + d * d); R[1] = 2.0 * (b * c - a * d);       R[2] = 2.0 * (b * d + a * c);
    R[3] = 2.0 * (b * c + a * d);       R[4] = 1.0 - 2.0 * (b * b + d * d); R[5] = 2.0 * (c * d - a * b);
    R[6] = 2.0 * (b * d - a * c);       R[7] = 2.0 * (c * d + a * b);       R[8] = 1.0 - 2.0 * (b * b + c * c);
}

static void project_one(int64_t i, const double *means, const double *quats, const double *log_scales,
                        const double *opacity_logits, const double *sh_color, const double *sh_weight,
                        double sigma, const ocam *cam, int W, int H, double bbox_slack, oproj *P) {
    memset(P, 0, sizeof(*P));
    const double *mu = means + 3 * i;
    /* camera-space centre */
    for (int r = 0; r < 3; ++r)
        P->t[r] = cam->R[3 * r + 0] * mu[0] + cam->R[3 * r + 1] * mu[1] + cam->R[3 * r + 2] * mu[2] + cam->t[r];
    P->o = 1.0 / (1.0 + exp(-opacity_logits[i]));
    if (P->t[2] <= OR_NEAR_Z || P->o < OR_ALPHA_MIN) { P->valid = 0; return; }
    P->valid = 1;
    const double x = P->t[0], y = P->t[1], z = P->t[2];
    P->m2[0] = cam->fx * x / z + cam->cx;
    P->m2[1] = cam->fy * y / z + cam->cy;

    /* Eq. 2: Sigma = R S S^T R^T */
    const double *q = quats + 4 * i;
    P->qlen = sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
    for (int k = 0; k < 4; ++k) P->qn[k] = q[k] / P->qlen;
    quat_to_rot(P->qn, P->Rq);
    for (int k = 0; k < 3; ++k) P->s[k] = exp(log_scales[3 * i + k]);
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) {
            double acc = 0.0;
            for (int k = 0; k < 3; ++k) acc += P->Rq[3 * a + k] * P->s[k] * P->s[k] * P->Rq[3 * b + k];
            P->Sig[3 * a + b] = acc;
        }

    /* Eq. 6: J (affine approximation of the projection at t), T = J W */
    P->J[0] = cam->fx / z; P->J[1] = 0.0;          P->J[2] = -cam->fx * x / (z * z);
    P->J[3] = 0.0;         P->J[4] = cam->fy / z;  P->J[5] = -cam->fy * y / (z * z);
    for (int a = 0; a < 2; ++a)
        for (int b = 0; b < 3; ++b) {
            double acc = 0.0;
            for (int k = 0; k < 3; ++k) acc += P->J[3 * a + k] * cam->R[3 * k + b];
            P->Tm[3 * a + b] = acc;
        }
    double C2[4];
    for (int a = 0; a < 2; ++a)
        for (int b = 0; b < 2; ++b) {
            double acc = 0.0;
            for (int k = 0; k < 3; ++k)
                for (int l = 0; l < 3; ++l) acc += P->Tm[3 * a + k] * P->Sig[3 * k + l] * P->Tm[3 * b + l];
            C2[2 * a + b] = acc;
        }
    P->cov[0] = C2[0] + OR_DILATION;
    P->cov[1] = 0.5 * (C2[1] + C2[2]);
    P->cov[2] = C2[3] + OR_DILATION;
    double det = P->cov[0] * P->cov[2] - P->cov[1] * P->cov[1];
    P->con[0] = P->cov[2] / det;
    P->con[1] = -P->cov[1] / det;
    P->con[2] = P->cov[0] / det;

    /* Eq. 4: view direction and SH colour; Eq. 1: OIT weight */
    double d[3];
    for (int k = 0; k < 3; ++k) d[k] = mu[k] - cam->pos[k];
    P->dlen = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
    for (int k = 0; k < 3; ++k) P->n[k] = d[k] / P->dlen;
    oracle_sh_basis(P->n, P->Y, NULL);
    const double *h = sh_color + 48 * i, *hw = sh_weight + 16 * i;
    for (int ch = 0; ch < 3; ++ch) {
        double acc = 0.0;
        for (int k = 0; k < 16; ++k) acc += P->Y[k] * h[3 * k + ch];
        P->c_raw[ch] = acc + 0.5;
        P->c[ch] = P->c_raw[ch] > 0.0 ? P->c_raw[ch] : 0.0;
    }
    double acc = 0.0;
    for (int k = 0; k < 16; ++k) acc += P->Y[k] * hw[k];
    P->v_raw = acc + 0.5;
    P->v = P->v_raw > 0.0 ? P->v_raw : 0.0;
    P->zterm = 1.0 - z / sigma;
    P->w = (P->zterm > 0.0 ? P->zterm : 0.0) * P->v;

    /* Pixel bbox of the ellipse {p <= ln(255 o)} where alpha can reach 1/255:
     * its half-extents are sqrt(2 ln(255 o) Sigma'_xx) and ... _yy.  The
     * threshold is raised by bbox_slack so that the box is a strict superset
     * (the per-pixel test below decides). */
    double lt = log(255.0 * P->o) + bbox_slack;
    double hx = sqrt(2.0 * lt * P->cov[0]) + 1e-9, hy = sqrt(2.0 * lt * P->cov[2]) + 1e-9;
    double fx0 = ceil(P->m2[0] - hx - 0.5), fx1 = floor(P->m2[0] + hx - 0.5);
    double fy0 = ceil(P->m2[1] - hy - 0.5), fy1 = floor(P->m2[1] + hy - 0.5);
    if (fx0 < 0) fx0 = 0;
    if (fy0 < 0) fy0 = 0;
    if (fx1 > W - 1) fx1 = W - 1;
    if (fy1 > H - 1) fy1 = H - 1;
    if (fx1 < fx0 || fy1 < fy0) { P->x0 = 0; P->x1 = -1; P->y0 = 0; P->y1 = -1; }
    else { P->x0 = (int)fx0; P->x1 = (int)fx1; P->y0 = (int)fy0; P->y1 = (int)fy1; }
}

/* Eq. 5 at pixel centre (px, py): returns the unclamped o exp(-p) and p. */
static inline double pair_alpha_raw(const oproj *P, double px, double py, double *dx_out, double *dy_out,
                                    double *p_out) {
    double dx = px - P->m2[0], dy = py - P->m2[1];
    double p = 0.5 * (P->con[0] * dx * dx + 2.0 * P->con[1] * dx * dy + P->con[2] * dy * dy);
    if (dx_out) *dx_out = dx;
    if (dy_out) *dy_out = dy;
    if (p_out) *p_out = p;
    return P->o * exp(-p);
}

static inline int near_log(double a, double b, double band) {
    return band > 0.0 && a > 0.0 && fabs(log(a) - log(b)) < band;
}

/* Projection of every splat; out[n, 24] (double), layout:
 *  0 valid, 1-2 mu', 3-5 Sigma' (xx, xy, yy), 6-8 conic, 9 o, 10-12 colour,
 *  13 v, 14 w, 15-17 camera-space centre, 18-20 unit view direction,
 *  21 1 - t_z/sigma, 22 ln(255 o), 23 unused. */
int oracle_project(int64_t n, const double *means, const double *quats, const double *log_scales,
                   const double *opacity_logits, const double *sh_color, const double *sh_weight,
                   double sigma, const double *cam_in, int W, int H, double *out) {
    ocam cam;
    load_camera(cam_in, &cam);
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) {
        oproj P;
        project_one(i, means, quats, log_scales, opacity_logits, sh_color, sh_weight, sigma, &cam, W, H, 0.0, &P);
        double *o = out + 24 * i;
        memset(o, 0, 24 * sizeof(double));
        o[0] = P.valid;
        o[9] = P.o;
        for (int k = 0; k < 3; ++k) o[15 + k] = P.t[k];
        if (!P.valid) continue;
        o[1] = P.m2[0]; o[2] = P.m2[1];
        for (int k = 0; k < 3; ++k) { o[3 + k] = P.cov[k]; o[6 + k] = P.con[k]; o[10 + k] = P.c[k]; o[18 + k] = P.n[k]; }
        o[13] = P.v; o[14] = P.w; o[21] = P.zterm; o[22] = log(255.0 * P.o);
    }
    return 0;
}

/* ---------------------------------------------------------- render ---- */

static void clip_window(const int *window, int W, int H, int *wx0, int *wy0, int *wx1, int *wy1) {
    *wx0 = 0; *wy0 = 0; *wx1 = W; *wy1 = H;
    if (window) {
        *wx0 = window[0] > 0 ? window[0] : 0;
        *wy0 = window[1] > 0 ? window[1] : 0;
        *wx1 = window[2] < W ? window[2] : W;
        *wy1 = window[3] < H ? window[3] : H;
    }
}

/* Per-pixel sums of the splats selected by `subset` (NULL = all):
 *   sums[0..2][HW] = P (sum of alpha w c), sums[3][HW] = Q (sum of alpha w),
 *   sums[4][HW] = log T (sum of log(1 - alpha)).
 * brute != 0 tests every splat at every pixel; otherwise each splat only
 * visits its pixel bbox (binned by 16-row bands).  Only pixels inside
 * `window` (x0, y0, x1, y1, half-open; NULL = whole view) are computed, the
 * rest of `sums` is zero.  amb_pixel (optional, [HW]) counts the pairs whose
 * unclamped alpha lies within a factor exp(amb_band) of the 1/255 threshold.
 * amb_sums (optional, [3][HW]) accumulates over those pairs sum a/(1 - a),
 * sum a w and sum a w max_c c (a = the unclamped alpha): enough to bound
 * how much adding or dropping them can move the composed colour.
 * stats (optional, [2]) = number of contributing (splat, pixel) pairs and of
 * pairs clamped at 0.99. */
int oracle_render_sums(int64_t n, const double *means, const double *quats, const double *log_scales,
                       const double *opacity_logits, const double *sh_color, const double *sh_weight,
                       double sigma, const double *cam_in, int W, int H, const uint8_t *subset, int brute,
                       const int *window, double amb_band, double *sums, int32_t *amb_pixel, int64_t *stats,
                       double *amb_sums) {
    ocam cam;
    load_camera(cam_in, &cam);
    const int64_t HW = (int64_t)W * H;
    memset(sums, 0, 5 * HW * sizeof(double));
    if (amb_pixel) memset(amb_pixel, 0, HW * sizeof(int32_t));
    if (amb_sums) memset(amb_sums, 0, 3 * HW * sizeof(double));
    int wx0, wy0, wx1, wy1;
    clip_window(window, W, H, &wx0, &wy0, &wx1, &wy1);
    if (wx1 <= wx0 || wy1 <= wy0) { if (stats) { stats[0] = 0; stats[1] = 0; } return 0; }

    oproj *proj = (oproj *)malloc((size_t)(n > 0 ? n : 1) * sizeof(oproj));
    if (!proj) return -1;
    double slack = (amb_band > 1e-6 ? amb_band : 1e-6) + 1e-9;
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) {
        if (subset && !subset[i]) { proj[i].valid = 0; continue; }
        project_one(i, means, quats, log_scales, opacity_logits, sh_color, sh_weight, sigma, &cam, W, H, slack,
                    &proj[i]);
    }

    /* bins of 16 rows: splat lists in ascending index */
    const int nb = (H + OR_BAND - 1) / OR_BAND;
    int64_t *cnt = (int64_t *)calloc((size_t)nb + 1, sizeof(int64_t));
    int64_t *lists = NULL;
    if (!brute) {
        for (int64_t i = 0; i < n; ++i) {
            const oproj *P = &proj[i];
            if (!P->valid || P->x1 < P->x0) continue;
            for (int b = P->y0 / OR_BAND; b <= P->y1 / OR_BAND; ++b) cnt[b + 1]++;
        }
        for (int b = 0; b < nb; ++b) cnt[b + 1] += cnt[b];
        lists = (int64_t *)malloc((size_t)(cnt[nb] > 0 ? cnt[nb] : 1) * sizeof(int64_t));
        int64_t *fill = (int64_t *)malloc((size_t)nb * sizeof(int64_t));
        for (int b = 0; b < nb; ++b) fill[b] = cnt[b];
        for (int64_t i = 0; i < n; ++i) {
            const oproj *P = &proj[i];
            if (!P->valid || P->x1 < P->x0) continue;
            for (int b = P->y0 / OR_BAND; b <= P->y1 / OR_BAND; ++b) lists[fill[b]++] = i;
        }
        free(fill);
    }

    int64_t n_pairs = 0, n_clamped = 0;
#pragma omp parallel for schedule(dynamic, 1) reduction(+ : n_pairs, n_clamped)
    for (int y = wy0; y < wy1; ++y) {
        const int b = y / OR_BAND;
        const int64_t lo = brute ? 0 : cnt[b], hi = brute ? n : cnt[b + 1];
        for (int x = wx0; x < wx1; ++x) {
            const int64_t pix = (int64_t)y * W + x;
            const double px = x + 0.5, py = y + 0.5;
            double Pr = 0, Pg = 0, Pb = 0, Q = 0, lT = 0;
            double ab0 = 0, ab1 = 0, ab2 = 0;
            int amb = 0;
            for (int64_t e = lo; e < hi; ++e) {
                const int64_t i = brute ? e : lists[e];
                const oproj *P = &proj[i];
                if (!P->valid) continue;
                if (!brute && (x < P->x0 || x > P->x1 || y < P->y0 || y > P->y1)) continue;
                double ar = pair_alpha_raw(P, px, py, NULL, NULL, NULL);
                if (near_log(ar, OR_ALPHA_MIN, amb_band)) {
                    amb++;
                    double cm = P->c[0] > P->c[1] ? P->c[0] : P->c[1];
                    cm = cm > P->c[2] ? cm : P->c[2];
                    ab0 += ar / (1.0 - ar);
                    ab1 += ar * P->w;
                    ab2 += ar * P->w * cm;
                }
                if (ar < OR_ALPHA_MIN) continue;
                double a = ar < OR_ALPHA_MAX ? ar : OR_ALPHA_MAX;
                if (ar > OR_ALPHA_MAX) n_clamped++;
                n_pairs++;
                double aw = a * P->w;
                Pr += aw * P->c[0];
                Pg += aw * P->c[1];
                Pb += aw * P->c[2];
                Q += aw;
                lT += log1p(-a);
            }
            sums[0 * HW + pix] = Pr;
            sums[1 * HW + pix] = Pg;
            sums[2 * HW + pix] = Pb;
            sums[3 * HW + pix] = Q;
            sums[4 * HW + pix] = lT;
            if (amb_pixel) amb_pixel[pix] = amb;
            if (amb_sums) {
                amb_sums[0 * HW + pix] = ab0;
                amb_sums[1 * HW + pix] = ab1;
                amb_sums[2 * HW + pix] = ab2;
            }
        }
    }
    if (stats) { stats[0] = n_pairs; stats[1] = n_clamped; }
    free(lists);
    free(cnt);
    free(proj);
    return 0;
}

/* Eq. 7 / Eq. 9 from the sums: T = exp(log T), F = P/Q (0 if Q = 0),
 * C = T c0 + (1 - T) F.  image[HW*3] (HWC).  aux (optional, [HW*5]) gets
 * (F_r, F_g, F_b, T, Q) per pixel. */
int oracle_compose(int W, int H, const double *sums, const double *bg, double *image, double *aux) {
    const int64_t HW = (int64_t)W * H;
    for (int64_t p = 0; p < HW; ++p) {
        double Q = sums[3 * HW + p];
        double T = exp(sums[4 * HW + p]);
        for (int ch = 0; ch < 3; ++ch) {
            double F = Q > 0.0 ? sums[ch * HW + p] / Q : 0.0;
            image[3 * p + ch] = T * bg[ch] + (1.0 - T) * F;
            if (aux) aux[5 * p + ch] = F;
        }
        if (aux) { aux[5 * p + 3] = T; aux[5 * p + 4] = Q; }
    }
    return 0;
}

/* -------------------------------------------------------- backward ---- */

/* Screen-space accumulators of one splat: dL/dmu' (2), dL/dK (K00, K01 = K10,
 * K11), dL/do, dL/dc (3), dL/dw. */
typedef struct {
    double m2[2], K[3], o, c[3], w;
} screen_grads;

/* Eq. 10 contracted with g = dL/dC at one pixel (state T, F, Q), for the pair
 * with unclamped alpha ar at offset (dx, dy), exponent p; added to *sg.
 * The alpha path (o, mu', K) is skipped where alpha is clamped at 0.99. */
static void pair_screen_grads(const oproj *P, double ar, double dx, double dy, double p, double T, const double F[3],
                              double Q, const double g[3], const double *bg, screen_grads *sg) {
    double a = ar < OR_ALPHA_MAX ? ar : OR_ALPHA_MAX;
    double invQ = Q > 0.0 ? 1.0 / Q : 0.0;
    double dLda = 0.0, dLdw = 0.0;
    for (int ch = 0; ch < 3; ++ch) {
        double dCdc = (1.0 - T) * a * P->w * invQ;
        double dCda = T / (1.0 - a) * (F[ch] - bg[ch]) + (1.0 - T) * P->w * invQ * (P->c[ch] - F[ch]);
        double dCdw = (1.0 - T) * a * invQ * (P->c[ch] - F[ch]);
        sg->c[ch] += g[ch] * dCdc;
        dLda += g[ch] * dCda;
        dLdw += g[ch] * dCdw;
    }
    sg->w += dLdw;
    if (ar <= OR_ALPHA_MAX) {
        /* a = o exp(-p): da/do = exp(-p), da/dp = -a;
         * p = 1/2 d^T K d: dp/dmu' = -K d, dp/dK = 1/2 d d^T */
        sg->o += dLda * exp(-p);
        double dLdp = -dLda * a;
        sg->m2[0] += dLdp * -(P->con[0] * dx + P->con[1] * dy);
        sg->m2[1] += dLdp * -(P->con[1] * dx + P->con[2] * dy);
        sg->K[0] += dLdp * 0.5 * dx * dx;
        sg->K[1] += dLdp * 0.5 * dx * dy;
        sg->K[2] += dLdp * 0.5 * dy * dy;
    }
}

/* Chain the screen-space gradients of splat P to its 75 parameters (gout,
 * overwritten) and to sigma (*dsig, overwritten): Eq. 6 (EWA projection and
 * the inverse), Eq. 1 (weight), Eq. 4 (SH colour / weight and the view
 * direction), Sec. 3.1 (sigmoid opacity), Eq. 2 (covariance from quaternion
 * and scales). */
static void chain_to_params(const oproj *P, const ocam *cam, const double *h, const double *hw, double sigma,
                            const screen_grads *sg, double *gout, double *dsig) {
    memset(gout, 0, OR_NPARAM * sizeof(double));
    *dsig = 0.0;
    /* K = Sigma'^-1: dL/dSigma' = -K G K with G the symmetric gradient in K */
    const double K[4] = {P->con[0], P->con[1], P->con[1], P->con[2]};
    const double G[4] = {sg->K[0], sg->K[1], sg->K[1], sg->K[2]};
    double KG[4], Gs[4];
    for (int a = 0; a < 2; ++a)
        for (int b = 0; b < 2; ++b) KG[2 * a + b] = K[2 * a + 0] * G[0 * 2 + b] + K[2 * a + 1] * G[1 * 2 + b];
    for (int a = 0; a < 2; ++a)
        for (int b = 0; b < 2; ++b) Gs[2 * a + b] = -(KG[2 * a + 0] * K[0 * 2 + b] + KG[2 * a + 1] * K[1 * 2 + b]);
    /* Sigma' = T Sigma T^T + 0.3 I, T = J W:
     *   dL/dSigma = T^T Gs T,  dL/dT = 2 Gs T Sigma */
    double gSig[9], gT[6];
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) {
            double acc = 0.0;
            for (int k = 0; k < 2; ++k)
                for (int l = 0; l < 2; ++l) acc += P->Tm[3 * k + a] * Gs[2 * k + l] * P->Tm[3 * l + b];
            gSig[3 * a + b] = acc;
        }
    for (int a = 0; a < 2; ++a)
        for (int b = 0; b < 3; ++b) {
            double acc = 0.0;
            for (int k = 0; k < 2; ++k)
                for (int l = 0; l < 3; ++l) acc += 2.0 * Gs[2 * a + k] * P->Tm[3 * k + l] * P->Sig[3 * l + b];
            gT[3 * a + b] = acc;
        }
    /* T = J W: dL/dJ = dL/dT W^T */
    double gJ[6];
    for (int a = 0; a < 2; ++a)
        for (int b = 0; b < 3; ++b) {
            double acc = 0.0;
            for (int k = 0; k < 3; ++k) acc += gT[3 * a + k] * cam->R[3 * b + k];
            gJ[3 * a + b] = acc;
        }
    const double x = P->t[0], y = P->t[1], z = P->t[2], fx = cam->fx, fy = cam->fy;
    double gt[3] = {0, 0, 0};
    /* J entries as functions of t */
    gt[0] += gJ[2] * (-fx / (z * z));
    gt[1] += gJ[5] * (-fy / (z * z));
    gt[2] += gJ[0] * (-fx / (z * z)) + gJ[2] * (2.0 * fx * x / (z * z * z)) + gJ[4] * (-fy / (z * z)) +
             gJ[5] * (2.0 * fy * y / (z * z * z));
    /* mu' = (fx x/z + cx, fy y/z + cy) */
    gt[0] += sg->m2[0] * fx / z;
    gt[1] += sg->m2[1] * fy / z;
    gt[2] += -sg->m2[0] * fx * x / (z * z) - sg->m2[1] * fy * y / (z * z);
    /* Eq. 1: w = max(0, 1 - z/sigma) v */
    double g_v = 0.0;
    if (P->zterm > 0.0) {
        g_v = sg->w * P->zterm;
        gt[2] += sg->w * P->v * (-1.0 / sigma);
        *dsig = sg->w * P->v * z / (sigma * sigma);
    }
    /* Eq. 4 colour and weight SH */
    double Yb[16], dY[48];
    oracle_sh_basis(P->n, Yb, dY);
    double g_n[3] = {0, 0, 0};
    for (int ch = 0; ch < 3; ++ch) {
        if (!(P->c_raw[ch] > 0.0)) continue;
        for (int k = 0; k < 16; ++k) {
            gout[11 + 3 * k + ch] = sg->c[ch] * Yb[k];
            for (int e = 0; e < 3; ++e) g_n[e] += sg->c[ch] * h[3 * k + ch] * dY[3 * k + e];
        }
    }
    if (P->v_raw > 0.0) {
        for (int k = 0; k < 16; ++k) {
            gout[59 + k] = g_v * Yb[k];
            for (int e = 0; e < 3; ++e) g_n[e] += g_v * hw[k] * dY[3 * k + e];
        }
    }
    /* mean: t = R_w mu + t_w, n = (mu - pos)/|mu - pos| */
    double ndot = P->n[0] * g_n[0] + P->n[1] * g_n[1] + P->n[2] * g_n[2];
    for (int e = 0; e < 3; ++e) {
        double acc = cam->R[0 * 3 + e] * gt[0] + cam->R[1 * 3 + e] * gt[1] + cam->R[2 * 3 + e] * gt[2];
        acc += (g_n[e] - P->n[e] * ndot) / P->dlen;
        gout[e] = acc;
    }
    /* opacity: o = sigmoid(l) */
    gout[10] = sg->o * P->o * (1.0 - P->o);
    /* Eq. 2: Sigma = M M^T, M = R S: dL/dM = 2 dL/dSigma M */
    double M[9], gM[9];
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) M[3 * a + b] = P->Rq[3 * a + b] * P->s[b];
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) {
            double acc = 0.0;
            for (int k = 0; k < 3; ++k) acc += (gSig[3 * a + k] + gSig[3 * k + a]) * M[3 * k + b];
            gM[3 * a + b] = acc;
        }
    double gR[9];
    for (int b = 0; b < 3; ++b) {
        double gs = 0.0;
        for (int a = 0; a < 3; ++a) {
            gs += gM[3 * a + b] * P->Rq[3 * a + b];
            gR[3 * a + b] = gM[3 * a + b] * P->s[b];
        }
        gout[7 + b] = gs * P->s[b];
    }
    /* R(q^): partial derivatives of each entry in (a, b, c, d) = (w, x, y, z) */
    const double qa = P->qn[0], qb = P->qn[1], qc = P->qn[2], qd = P->qn[3];
    double gq[4] = {0, 0, 0, 0};
    /* R00 = 1 - 2(c^2 + d^2) */
    gq[2] += gR[0] * (-4.0 * qc); gq[3] += gR[0] * (-4.0 * qd);
    /* R01 = 2(bc - ad) */
    gq[0] += gR[1] * (-2.0 * qd); gq[1] += gR[1] * (2.0 * qc); gq[2] += gR[1] * (2.0 * qb); gq[3] += gR[1] * (-2.0 * qa);
    /* R02 = 2(bd + ac) */
    gq[0] += gR[2] * (2.0 * qc); gq[1] += gR[2] * (2.0 * qd); gq[2] += gR[2] * (2.0 * qa); gq[3] += gR[2] * (2.0 * qb);
    /* R10 = 2(bc + ad) */
    gq[0] += gR[3] * (2.0 * qd); gq[1] += gR[3] * (2.0 * qc); gq[2] += gR[3] * (2.0 * qb); gq[3] += gR[3] * (2.0 * qa);
    /* R11 = 1 - 2(b^2 + d^2) */
    gq[1] += gR[4] * (-4.0 * qb); gq[3] += gR[4] * (-4.0 * qd);
    /* R12 = 2(cd - ab) */
    gq[0] += gR[5] * (-2.0 * qb); gq[1] += gR[5] * (-2.0 * qa); gq[2] += gR[5] * (2.0 * qd); gq[3] += gR[5] * (2.0 * qc);
    /* R20 = 2(bd - ac) */
    gq[0] += gR[6] * (-2.0 * qc); gq[1] += gR[6] * (2.0 * qd); gq[2] += gR[6] * (-2.0 * qa); gq[3] += gR[6] * (2.0 * qb);
    /* R21 = 2(cd + ab) */
    gq[0] += gR[7] * (2.0 * qb); gq[1] += gR[7] * (2.0 * qa); gq[2] += gR[7] * (2.0 * qd); gq[3] += gR[7] * (2.0 * qc);
    /* R22 = 1 - 2(b^2 + c^2) */
    gq[1] += gR[8] * (-4.0 * qb); gq[2] += gR[8] * (-4.0 * qc);
    /* q^ = q / |q| */
    double qdot = qa * gq[0] + qb * gq[1] + qc * gq[2] + qd * gq[3];
    for (int k = 0; k < 4; ++k) gout[3 + k] = (gq[k] - P->qn[k] * qdot) / P->qlen;
}

/* Gradient of L = sum_pixels dL_dC . C with respect to every parameter of
 * the splats selected by `active` (NULL = all), for the image composed from
 * `sums_total` (the sums of ALL splats, e.g. active + frozen).  Only pixels
 * inside `window` contribute (dL_dC is read there only).
 *
 * grads[n, 75] rows of selected splats are overwritten, the others are not
 * touched.  Row layout: mean (3), quaternion (4), log-scale (3),
 * opacity logit (1), colour SH [16][3] (48), weight SH (16).
 * dsigma (optional, [3]) = dL/dsigma summed over the selected splats, the
 * sum of the absolute values of those per-splat terms (the scale a rounding
 * error of the sum is measured against), and the allowance of the near-cut
 * pairs for dL/dsigma (see flip).
 * amb_splat (optional, [n]) for a selected splat: bit 0 set if a pair's
 * unclamped alpha is within exp(amb_band) of 1/255 or of 0.99; bit 1 set if
 * a colour / weight SH value is within amb_band of the max(0,.) kink,
 * |1 - t_z/sigma| < amb_band or |t_z - 0.2| < amb_band (near plane).
 * flip (optional, [n, 75]) for a selected splat: the sum over its bit-0
 * pairs of |the parameter gradient of that pair alone| (each taken as
 * included and unclamped) -- how far a different inclusion / clamping
 * decision on those pairs can move its gradient.
 *
 * Per pair the derivatives of Eq. 10 are used as printed:
 *   dC/dc_i     = (1-T) a_i w_i / Q
 *   dC/da_i     = T/(1-a_i) (F - c0) + (1-T) (w_i/Q) (c_i - F)
 *   dC/dw_i     = (1-T) (a_i/Q) (c_i - F)
 * with the terms carrying 1/Q taken as 0 where Q = 0. */
int oracle_backward(int64_t n, const double *means, const double *quats, const double *log_scales,
                    const double *opacity_logits, const double *sh_color, const double *sh_weight, double sigma,
                    const double *bg, const double *cam_in, int W, int H, const uint8_t *active,
                    const double *sums_total, const double *dL_dC, const int *window, double amb_band,
                    double *grads, double *dsigma, uint8_t *amb_splat, double *flip) {
    ocam cam;
    load_camera(cam_in, &cam);
    const int64_t HW = (int64_t)W * H;
    int wx0, wy0, wx1, wy1;
    clip_window(window, W, H, &wx0, &wy0, &wx1, &wy1);
    double slack = (amb_band > 1e-6 ? amb_band : 1e-6) + 1e-9;
    double dsig_total = 0.0, dsig_abs = 0.0, dsig_flip = 0.0;

#pragma omp parallel for schedule(dynamic, 64) reduction(+ : dsig_total, dsig_abs, dsig_flip)
    for (int64_t i = 0; i < n; ++i) {
        if (active && !active[i]) continue;
        double *gout = grads + (int64_t)OR_NPARAM * i;
        double *fout = flip ? flip + (int64_t)OR_NPARAM * i : NULL;
        memset(gout, 0, OR_NPARAM * sizeof(double));
        if (fout) memset(fout, 0, OR_NPARAM * sizeof(double));
        if (amb_splat) amb_splat[i] = 0;
        oproj P;
        project_one(i, means, quats, log_scales, opacity_logits, sh_color, sh_weight, sigma, &cam, W, H, slack, &P);
        int amb = 0;
        if (amb_band > 0.0 && fabs(P.t[2] - OR_NEAR_Z) < amb_band) amb |= 2;
        if (!P.valid) {
            if (amb_splat) amb_splat[i] = (uint8_t)amb;
            continue;
        }
        if (amb_band > 0.0) {
            for (int ch = 0; ch < 3; ++ch) if (fabs(P.c_raw[ch]) < amb_band) amb |= 2;
            if (fabs(P.v_raw) < amb_band || fabs(P.zterm) < amb_band) amb |= 2;
        }
        const double *h = sh_color + 48 * i, *hw = sh_weight + 16 * i;
        screen_grads sg;
        memset(&sg, 0, sizeof(sg));
        int x0 = P.x0 > wx0 ? P.x0 : wx0, x1 = P.x1 < wx1 - 1 ? P.x1 : wx1 - 1;
        int y0 = P.y0 > wy0 ? P.y0 : wy0, y1 = P.y1 < wy1 - 1 ? P.y1 : wy1 - 1;
        for (int y = y0; y <= y1; ++y) {
            for (int x = x0; x <= x1; ++x) {
                double dx, dy, p;
                double ar = pair_alpha_raw(&P, x + 0.5, y + 0.5, &dx, &dy, &p);
                const int near = near_log(ar, OR_ALPHA_MIN, amb_band) || near_log(ar, OR_ALPHA_MAX, amb_band);
                if (ar < OR_ALPHA_MIN && !near) continue;
                const int64_t pix = (int64_t)y * W + x;
                double Q = sums_total[3 * HW + pix];
                double T = exp(sums_total[4 * HW + pix]);
                double F[3], g[3];
                for (int ch = 0; ch < 3; ++ch) {
                    F[ch] = Q > 0.0 ? sums_total[ch * HW + pix] / Q : 0.0;
                    g[ch] = dL_dC[3 * pix + ch];
                }
                if (ar >= OR_ALPHA_MIN) pair_screen_grads(&P, ar, dx, dy, p, T, F, Q, g, bg, &sg);
                if (near) {
                    amb |= 1;
                    if (fout) {
                        /* this pair alone, taken as included and unclamped */
                        screen_grads one;
                        memset(&one, 0, sizeof(one));
                        double ar1 = ar < OR_ALPHA_MAX ? (ar > OR_ALPHA_MIN ? ar : OR_ALPHA_MIN) : OR_ALPHA_MAX;
                        pair_screen_grads(&P, ar1, dx, dy, p, T, F, Q, g, bg, &one);
                        double g1[OR_NPARAM], s1;
                        chain_to_params(&P, &cam, h, hw, sigma, &one, g1, &s1);
                        for (int k = 0; k < OR_NPARAM; ++k) fout[k] += fabs(g1[k]);
                        dsig_flip += fabs(s1);
                    }
                }
            }
        }
        if (amb_splat) amb_splat[i] = (uint8_t)amb;
        double ds;
        chain_to_params(&P, &cam, h, hw, sigma, &sg, gout, &ds);
        dsig_total += ds;
        dsig_abs += fabs(ds);
    }
    if (dsigma) { dsigma[0] = dsig_total; dsigma[1] = dsig_abs; dsigma[2] = dsig_flip; }
    return 0;
}

int oracle_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
