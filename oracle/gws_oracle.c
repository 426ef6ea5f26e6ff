/*
 * gws_oracle.c -- plain FP64 CPU oracle for Gaussian Wave Splatting
 * (Choi et al., "Gaussian Wave Splatting for Computer-Generated Holography",
 * arXiv 2505.06582).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the benchmark's CPU
 * baseline may load this file.  It shares no code, header, table or constant with the
 * CUDA library: it is the slow, obviously correct statement of what that library must
 * compute.  Every loop is the textbook definition: no truncation, no tiling, no
 * anchoring, no reordering beyond the sums the definitions state.
 *
 * Conventions (each one is a reading of the paper; the reasons are listed with the
 * design notes):
 *   - ordinary spatial frequency f = (fx, fy, fz) in cycles/m, fz = sqrt(1/lam^2 - fx^2
 *     - fy^2) inside the circle fx^2 + fy^2 < 1/lam^2 and no contribution outside
 *     (angular-spectrum transfer function, Eq. 4, Sec. 4);
 *   - centred grids: column c has fx = (c - floor(W/2)) / (W px), row r has
 *     fy = (r - floor(H/2)) / (H py); pixel (r, c) of the field sits at
 *     x = (c - floor(W/2)) px, y = (r - floor(H/2)) py;
 *   - quaternion q = (w, x, y, z), normalised here; R = [r1 r2 r3] (columns), r1 = t_u,
 *     r2 = t_v, r3 = normal (Sec. 3);
 *   - one Gaussian's angular spectrum at the SLM (Eq. 9-10, the supplement's
 *     translation / rotation / scaling derivation), with the on-axis reference wave
 *     f_r = (0, 0, 1/lam) shifting the spectrum (Sec. 4.1, last paragraph):
 *        u_i(f) = 2 pi s_u s_v |r3.f| / fz
 *                 * exp(-2 pi^2 [ s_u^2 (r1.d)^2 + s_v^2 (r2.d)^2 ]),  d = f - f_r
 *                 * exp(-j 2 pi f.mu)      [xy shift and the propagation H(f, -mu_z)]
 *                 * (phase_match ? exp(+j 2 pi mu_z / lam) : 1)
 *   - blending: order-invariant sum (Eq. 12) with weight c o, or the depth-sorted
 *     variant with weight c o T_i, T_i = prod over front Gaussians of (1 - alpha_j(mu_i))
 *     (Eq. 5-6 with T held at the Gaussian's centre, alpha from Eq. 2, t_eps = 1/255 from
 *     Algorithm S2);
 *   - field = centred inverse DFT scaled by dfx dfy (continuous inverse transform of
 *     Eq. 3 sampled on the grid);
 *   - double-phase encoding (supplement, phase encoding): P1,2 = phi -/+ acos(a / a_max),
 *     checkerboard (r + c even -> P1), wrapped to [-pi, pi).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

#define TWO_PI 6.283185307179586476925286766559
#define PI 3.1415926535897932384626433832795

/* ------------------------------------------------------------------------------------ */
/* Gaussian geometry                                                                     */
/* ------------------------------------------------------------------------------------ */

/* Rotation matrix of the normalised quaternion; columns r1, r2, r3 (Hamilton, w first). */
static void rotation_columns(const double qin[4], double r1[3], double r2[3], double r3[3], double qhat[4],
                             double *qnorm) {
    double n = sqrt(qin[0] * qin[0] + qin[1] * qin[1] + qin[2] * qin[2] + qin[3] * qin[3]);
    double w = qin[0] / n, x = qin[1] / n, y = qin[2] / n, z = qin[3] / n;
    r1[0] = 1.0 - 2.0 * (y * y + z * z);
    r1[1] = 2.0 * (x * y + w * z);
    r1[2] = 2.0 * (x * z - w * y);
    r2[0] = 2.0 * (x * y - w * z);
    r2[1] = 1.0 - 2.0 * (x * x + z * z);
    r2[2] = 2.0 * (y * z + w * x);
    r3[0] = 2.0 * (x * z + w * y);
    r3[1] = 2.0 * (y * z - w * x);
    r3[2] = 1.0 - 2.0 * (x * x + y * y);
    if (qhat) {
        qhat[0] = w; qhat[1] = x; qhat[2] = y; qhat[3] = z;
    }
    if (qnorm) *qnorm = n;
}

static double dot3(const double a[3], const double b[3]) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }

typedef struct {
    double mu[3];
    double r1[3], r2[3], r3[3];
    double qhat[4], qnorm;
    double su, sv, o;
} gauss_t;

static void load_gaussian(int64_t i, const double *mean, const double *quat, const double *scale,
                          const double *opacity, gauss_t *g) {
    g->mu[0] = mean[3 * i]; g->mu[1] = mean[3 * i + 1]; g->mu[2] = mean[3 * i + 2];
    rotation_columns(quat + 4 * i, g->r1, g->r2, g->r3, g->qhat, &g->qnorm);
    g->su = scale[2 * i]; g->sv = scale[2 * i + 1];
    g->o = opacity[i];
}

/* ------------------------------------------------------------------------------------ */
/* Depth order (front = nearest the SLM = smallest z; ties -> lower input index first)   */
/* ------------------------------------------------------------------------------------ */

static const double *g_sort_z;
static int cmp_depth(const void *pa, const void *pb) {
    int64_t a = *(const int64_t *)pa, b = *(const int64_t *)pb;
    double za = g_sort_z[3 * a + 2], zb = g_sort_z[3 * b + 2];
    if (za < zb) return -1;
    if (za > zb) return 1;
    return (a < b) ? -1 : (a > b);
}

/* Writes the input indices in front-to-back order (Algorithm S2 sorts front to back). */
void gwso_depth_order(int64_t n, const double *mean, int64_t *order) {
    for (int64_t i = 0; i < n; ++i) order[i] = i;
    g_sort_z = mean;
    qsort(order, (size_t)n, sizeof(int64_t), cmp_depth);
}

/* ------------------------------------------------------------------------------------ */
/* Opacity footprint (Eq. 2) of Gaussian j at a point x of the hologram plane           */
/* ------------------------------------------------------------------------------------ */

/* alpha_j(x) = o_j exp(-1/2 |M^-1 (x - mu_j)_xy|^2), M = [s_u r1_xy, s_v r2_xy]: the
 * Gaussian's in-focus footprint projected along z (peak o_j at its centre).  An edge-on
 * Gaussian (|det M| < 1e-14 s_u s_v) has no footprint. */
static double alpha_at(const gauss_t *g, double x, double y) {
    double m00 = g->su * g->r1[0], m01 = g->sv * g->r2[0];
    double m10 = g->su * g->r1[1], m11 = g->sv * g->r2[1];
    double det = m00 * m11 - m01 * m10;
    if (fabs(det) < 1e-14 * g->su * g->sv) return 0.0;
    double dx = x - g->mu[0], dy = y - g->mu[1];
    double y0 = (m11 * dx - m01 * dy) / det;
    double y1 = (-m10 * dx + m00 * dy) / det;
    return g->o * exp(-0.5 * (y0 * y0 + y1 * y1));
}

/* Transmittance at each Gaussian's centre, T_i = prod_{j in front of i} (1 - alpha_j(mu_i)),
 * with alpha_j < alpha_min dropped (t_eps of Algorithm S2).  T is written per input index. */
void gwso_transmittance(int64_t n, const double *mean, const double *quat, const double *scale,
                        const double *opacity, double alpha_min, double *T) {
    int64_t *order = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
    gwso_depth_order(n, mean, order);
    gauss_t *gs = (gauss_t *)malloc(sizeof(gauss_t) * (size_t)(n > 0 ? n : 1));
    for (int64_t p = 0; p < n; ++p) load_gaussian(order[p], mean, quat, scale, opacity, &gs[p]);
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t p = 0; p < n; ++p) {
        double t = 1.0;
        for (int64_t q = 0; q < p; ++q) {
            double a = alpha_at(&gs[q], gs[p].mu[0], gs[p].mu[1]);
            if (a >= alpha_min) t *= (1.0 - a);
        }
        T[order[p]] = t;
    }
    free(gs);
    free(order);
}

/* Transmittance for a subset of Gaussians (input indices `which`), O(N) each. */
void gwso_transmittance_at(int64_t n, const double *mean, const double *quat, const double *scale,
                           const double *opacity, double alpha_min, int64_t n_which, const int64_t *which,
                           double *T) {
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t k = 0; k < n_which; ++k) {
        int64_t i = which[k];
        double xi = mean[3 * i], yi = mean[3 * i + 1], zi = mean[3 * i + 2];
        double t = 1.0;
        for (int64_t j = 0; j < n; ++j) {
            double zj = mean[3 * j + 2];
            int front = (zj < zi) || (zj == zi && j < i);
            if (!front) continue;
            gauss_t g;
            load_gaussian(j, mean, quat, scale, opacity, &g);
            double a = alpha_at(&g, xi, yi);
            if (a >= alpha_min) t *= (1.0 - a);
        }
        T[k] = t;
    }
}

/* ------------------------------------------------------------------------------------ */
/* Angular spectrum of one Gaussian (Eq. 10) at one grid frequency                      */
/* ------------------------------------------------------------------------------------ */

typedef struct {
    double fx, fy, fz, inv_lam;
    int propagating;
} freq_t;

static freq_t grid_freq(int r, int c, int H, int W, double px, double py, double lam) {
    freq_t f;
    f.fx = (double)(c - W / 2) / ((double)W * px);
    f.fy = (double)(r - H / 2) / ((double)H * py);
    f.inv_lam = 1.0 / lam;
    double rho2 = f.fx * f.fx + f.fy * f.fy;
    double k2 = f.inv_lam * f.inv_lam;
    f.propagating = rho2 < k2; /* strict inequality, Eq. 4 */
    f.fz = f.propagating ? sqrt(k2 - rho2) : 0.0;
    return f;
}

/* Unweighted spectrum u_i(f) (no colour, opacity, transmittance).  Also returns the
 * intermediate quantities the analytic gradient needs. */
typedef struct {
    double re, im;     /* u_i(f) */
    double a, b, g;    /* r1.d, r2.d, r3.f */
    double gauss;      /* exp(-2 pi^2 (su^2 a^2 + sv^2 b^2)) */
} term_t;

static term_t gaussian_term(const gauss_t *G, const freq_t *f, int phase_match) {
    term_t t;
    memset(&t, 0, sizeof t);
    if (!f->propagating) return t;
    double fv[3] = {f->fx, f->fy, f->fz};
    double d[3] = {f->fx, f->fy, f->fz - f->inv_lam}; /* d = f - f_r */
    t.a = dot3(G->r1, d);
    t.b = dot3(G->r2, d);
    t.g = dot3(G->r3, fv);
    t.gauss = exp(-2.0 * PI * PI * (G->su * G->su * t.a * t.a + G->sv * G->sv * t.b * t.b));
    double amp = TWO_PI * G->su * G->sv * fabs(t.g) / f->fz * t.gauss;
    /* phase in cycles: -f.mu (+ mu_z / lam); reduced to [-1/2, 1/2] before the 2 pi */
    double cyc = -(f->fx * G->mu[0] + f->fy * G->mu[1] + f->fz * G->mu[2]);
    if (phase_match) cyc += G->mu[2] * f->inv_lam;
    cyc -= nearbyint(cyc);
    t.re = amp * cos(TWO_PI * cyc);
    t.im = amp * sin(TWO_PI * cyc);
    return t;
}

/* Neumaier-compensated complex accumulator */
typedef struct { double s[2], c[2]; } acc_t;
static void acc_add1(double *s, double *c, double x) {
    double t = *s + x;
    if (fabs(*s) >= fabs(x)) *c += (*s - t) + x;
    else *c += (x - t) + *s;
    *s = t;
}
static void acc_add(acc_t *a, double re, double im) {
    acc_add1(&a->s[0], &a->c[0], re);
    acc_add1(&a->s[1], &a->c[1], im);
}

/* Per-Gaussian blending weights w[i][l] = c_il o_i T_i (T = 1 for the order-invariant sum). */
static double *blend_weights(int64_t n, const double *mean, const double *quat, const double *scale,
                             const double *opacity, const double *amp, int n_lambda, int blend,
                             double alpha_min) {
    double *w = (double *)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1) * (size_t)n_lambda);
    double *T = (double *)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    for (int64_t i = 0; i < n; ++i) T[i] = 1.0;
    if (blend == 1) gwso_transmittance(n, mean, quat, scale, opacity, alpha_min, T);
    for (int64_t i = 0; i < n; ++i)
        for (int l = 0; l < n_lambda; ++l) w[i * n_lambda + l] = amp[i * n_lambda + l] * opacity[i] * T[i];
    free(T);
    return w;
}

/* Full spectrum u_SLM(f) = sum_i w_i u_i(f) (Eq. 12, or Eq. 5 with T at the centre),
 * summed front to back.  out: complex128 interleaved [n_lambda][H][W]. */
void gwso_spectrum(int64_t n, const double *mean, const double *quat, const double *scale,
                   const double *opacity, const double *amp, int n_lambda, const double *wavelengths, int H,
                   int W, double px, double py, int blend, int phase_match, double alpha_min, double *out) {
    int64_t *order = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
    gwso_depth_order(n, mean, order);
    double *w = blend_weights(n, mean, quat, scale, opacity, amp, n_lambda, blend, alpha_min);
    gauss_t *gs = (gauss_t *)malloc(sizeof(gauss_t) * (size_t)(n > 0 ? n : 1));
    for (int64_t p = 0; p < n; ++p) load_gaussian(order[p], mean, quat, scale, opacity, &gs[p]);
    for (int l = 0; l < n_lambda; ++l) {
#pragma omp parallel for schedule(dynamic, 1)
        for (int r = 0; r < H; ++r) {
            for (int c = 0; c < W; ++c) {
                freq_t f = grid_freq(r, c, H, W, px, py, wavelengths[l]);
                acc_t acc;
                memset(&acc, 0, sizeof acc);
                for (int64_t p = 0; p < n; ++p) {
                    term_t t = gaussian_term(&gs[p], &f, phase_match);
                    double wi = w[order[p] * n_lambda + l];
                    acc_add(&acc, wi * t.re, wi * t.im);
                }
                size_t o = ((size_t)l * H + r) * W + c;
                out[2 * o] = acc.s[0] + acc.c[0];
                out[2 * o + 1] = acc.s[1] + acc.c[1];
            }
        }
    }
    free(gs);
    free(w);
    free(order);
}

/* The same spectrum at selected samples (lambda index, row, column); O(N) per sample.
 * T_in: optional per-Gaussian transmittance (NULL -> 1, i.e. the order-invariant sum). */
void gwso_spectrum_at(int64_t n, const double *mean, const double *quat, const double *scale,
                      const double *opacity, const double *amp, const double *T_in, int n_lambda,
                      const double *wavelengths, int H, int W, double px, double py, int phase_match,
                      int64_t n_samples, const int32_t *s_lam, const int32_t *s_row, const int32_t *s_col,
                      double *out) {
    int64_t *order = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
    gwso_depth_order(n, mean, order);
    gauss_t *gs = (gauss_t *)malloc(sizeof(gauss_t) * (size_t)(n > 0 ? n : 1));
    for (int64_t p = 0; p < n; ++p) load_gaussian(order[p], mean, quat, scale, opacity, &gs[p]);
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t k = 0; k < n_samples; ++k) {
        int l = s_lam[k];
        freq_t f = grid_freq(s_row[k], s_col[k], H, W, px, py, wavelengths[l]);
        acc_t acc;
        memset(&acc, 0, sizeof acc);
        for (int64_t p = 0; p < n; ++p) {
            int64_t i = order[p];
            term_t t = gaussian_term(&gs[p], &f, phase_match);
            double wi = amp[i * n_lambda + l] * opacity[i] * (T_in ? T_in[i] : 1.0);
            acc_add(&acc, wi * t.re, wi * t.im);
        }
        out[2 * k] = acc.s[0] + acc.c[0];
        out[2 * k + 1] = acc.s[1] + acc.c[1];
    }
    free(gs);
    free(order);
}

/* Per-pixel factors of one Gaussian at one wavelength: the unweighted spectrum (complex)
 * and the Gaussian exponent E = 2 pi^2 (su^2 a^2 + sv^2 b^2).  out_term: complex [H][W],
 * out_E: [H][W]. */
void gwso_single_terms(const double *mean3, const double *quat4, const double *scale2, double lam, int H,
                       int W, double px, double py, int phase_match, double *out_term, double *out_E) {
    gauss_t G;
    double one = 1.0;
    load_gaussian(0, mean3, quat4, scale2, &one, &G);
    for (int r = 0; r < H; ++r)
        for (int c = 0; c < W; ++c) {
            freq_t f = grid_freq(r, c, H, W, px, py, lam);
            term_t t = gaussian_term(&G, &f, phase_match);
            size_t o = (size_t)r * W + c;
            out_term[2 * o] = t.re;
            out_term[2 * o + 1] = t.im;
            out_E[o] = f.propagating ? 2.0 * PI * PI * (G.su * G.su * t.a * t.a + G.sv * G.sv * t.b * t.b)
                                     : INFINITY;
        }
}

/* ------------------------------------------------------------------------------------ */
/* Centred inverse DFT (Eq. 3 sampled on the grid) and its adjoint                      */
/* ------------------------------------------------------------------------------------ */

/* exp(sign * j 2 pi k / N) for k = 0..N-1, exact integer reduction of the angle index */
static double *twiddles(int N, int sign) {
    double *t = (double *)malloc(sizeof(double) * 2 * (size_t)N);
    for (int k = 0; k < N; ++k) {
        t[2 * k] = cos(TWO_PI * (double)k / (double)N);
        t[2 * k + 1] = sign * sin(TWO_PI * (double)k / (double)N);
    }
    return t;
}
static int modidx(int64_t a, int N) {
    int64_t m = a % N;
    return (int)(m < 0 ? m + N : m);
}

/* out[r][c] = scale * sum_m sum_n in[m][n] exp(sign j 2 pi ((m-m0)(r-r0)/H + (n-n0)(c-c0)/W)),
 * m0 = r0 = floor(H/2), n0 = c0 = floor(W/2); separable direct sums, rows then columns. */
static void centred_dft2(const double *in, double *out, int H, int W, int sign, double scale) {
    double *tw_w = twiddles(W, sign), *tw_h = twiddles(H, sign);
    double *tmp = (double *)malloc(sizeof(double) * 2 * (size_t)H * W);
    int m0 = H / 2, n0 = W / 2;
#pragma omp parallel for schedule(static)
    for (int m = 0; m < H; ++m)
        for (int c = 0; c < W; ++c) {
            double sr = 0, si = 0;
            for (int nn = 0; nn < W; ++nn) {
                int k = modidx((int64_t)(nn - n0) * (c - n0), W);
                double xr = in[2 * ((size_t)m * W + nn)], xi = in[2 * ((size_t)m * W + nn) + 1];
                sr += xr * tw_w[2 * k] - xi * tw_w[2 * k + 1];
                si += xr * tw_w[2 * k + 1] + xi * tw_w[2 * k];
            }
            tmp[2 * ((size_t)m * W + c)] = sr;
            tmp[2 * ((size_t)m * W + c) + 1] = si;
        }
#pragma omp parallel for schedule(static)
    for (int r = 0; r < H; ++r)
        for (int c = 0; c < W; ++c) {
            double sr = 0, si = 0;
            for (int m = 0; m < H; ++m) {
                int k = modidx((int64_t)(m - m0) * (r - m0), H);
                double xr = tmp[2 * ((size_t)m * W + c)], xi = tmp[2 * ((size_t)m * W + c) + 1];
                sr += xr * tw_h[2 * k] - xi * tw_h[2 * k + 1];
                si += xr * tw_h[2 * k + 1] + xi * tw_h[2 * k];
            }
            out[2 * ((size_t)r * W + c)] = scale * sr;
            out[2 * ((size_t)r * W + c) + 1] = scale * si;
        }
    free(tmp);
    free(tw_w);
    free(tw_h);
}

/* field = dfx dfy * centred inverse DFT of the spectrum (per wavelength slice).
 * spec, field: complex128 [n_slices][H][W]. */
void gwso_idft(int n_slices, int H, int W, double px, double py, const double *spec, double *field) {
    double dfx = 1.0 / (W * px), dfy = 1.0 / (H * py);
    for (int s = 0; s < n_slices; ++s)
        centred_dft2(spec + 2 * (size_t)s * H * W, field + 2 * (size_t)s * H * W, H, W, +1, dfx * dfy);
}

/* Adjoint of gwso_idft: spec_grad = dfx dfy * centred forward DFT (exp(-j ...)). */
void gwso_idft_adjoint(int n_slices, int H, int W, double px, double py, const double *field_grad,
                       double *spec_grad) {
    double dfx = 1.0 / (W * px), dfy = 1.0 / (H * py);
    for (int s = 0; s < n_slices; ++s)
        centred_dft2(field_grad + 2 * (size_t)s * H * W, spec_grad + 2 * (size_t)s * H * W, H, W, -1, dfx * dfy);
}

/* The inverse DFT at selected pixels only: O(H W) per pixel. */
void gwso_idft_at(int H, int W, double px, double py, const double *spec, int64_t n_samples,
                  const int32_t *s_row, const int32_t *s_col, double *out) {
    double dfx = 1.0 / (W * px), dfy = 1.0 / (H * py);
    double *tw_w = twiddles(W, +1), *tw_h = twiddles(H, +1);
    int m0 = H / 2, n0 = W / 2;
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t k = 0; k < n_samples; ++k) {
        int r = s_row[k], c = s_col[k];
        double sr = 0, si = 0;
        for (int m = 0; m < H; ++m) {
            int km = modidx((int64_t)(m - m0) * (r - m0), H);
            for (int nn = 0; nn < W; ++nn) {
                int kn = modidx((int64_t)(nn - n0) * (c - n0), W);
                double tr = tw_h[2 * km] * tw_w[2 * kn] - tw_h[2 * km + 1] * tw_w[2 * kn + 1];
                double ti = tw_h[2 * km] * tw_w[2 * kn + 1] + tw_h[2 * km + 1] * tw_w[2 * kn];
                double xr = spec[2 * ((size_t)m * W + nn)], xi = spec[2 * ((size_t)m * W + nn) + 1];
                sr += xr * tr - xi * ti;
                si += xr * ti + xi * tr;
            }
        }
        out[2 * k] = dfx * dfy * sr;
        out[2 * k + 1] = dfx * dfy * si;
    }
    free(tw_w);
    free(tw_h);
}

/* ------------------------------------------------------------------------------------ */
/* Double-phase amplitude encoding (supplement, phase encoding)                         */
/* ------------------------------------------------------------------------------------ */

static double wrap_pi(double x) { return x - TWO_PI * floor((x + PI) / TWO_PI); }

/* field: complex128 [n_lambda][H][W] -> phase [n_lambda][H][W].
 * a_max = max |u| per wavelength slice unless amp_scale > 0; amplitudes above a_max clamp
 * to 1.  Pixel (r, c) takes P1 = phi - acos(a) when r + c is even, else P2 = phi + acos(a). */
void gwso_encode(int n_lambda, int H, int W, const double *field, double amp_scale, double *phase) {
    for (int l = 0; l < n_lambda; ++l) {
        const double *u = field + 2 * (size_t)l * H * W;
        double amax = 0.0;
        if (amp_scale > 0) amax = amp_scale;
        else
            for (size_t k = 0; k < (size_t)H * W; ++k) {
                double m = hypot(u[2 * k], u[2 * k + 1]);
                if (m > amax) amax = m;
            }
        for (int r = 0; r < H; ++r)
            for (int c = 0; c < W; ++c) {
                size_t k = (size_t)r * W + c;
                double m = hypot(u[2 * k], u[2 * k + 1]);
                double a = amax > 0 ? m / amax : 0.0;
                if (a > 1.0) a = 1.0;
                double phi = atan2(u[2 * k + 1], u[2 * k]);
                double p = ((r + c) % 2 == 0) ? phi - acos(a) : phi + acos(a);
                phase[(size_t)l * H * W + k] = wrap_pi(p);
            }
    }
}

/* ------------------------------------------------------------------------------------ */
/* Analytic gradients                                                                    */
/* ------------------------------------------------------------------------------------ */

/* dL/dq from dL/dr1, dL/dr2, dL/dr3 through R(qhat) and qhat = q / |q|. */
static void quat_chain(const double qh[4], double qn, const double G1[3], const double G2[3], const double G3[3],
                       double dq[4]) {
    double w = qh[0], x = qh[1], y = qh[2], z = qh[3];
    /* d r_k / d qhat_m, written column by column */
    double dr1[4][3] = {{0, 2 * z, -2 * y}, {0, 2 * y, 2 * z}, {-4 * y, 2 * x, -2 * w}, {-4 * z, 2 * w, 2 * x}};
    double dr2[4][3] = {{-2 * z, 0, 2 * x}, {2 * y, -4 * x, 2 * w}, {2 * x, 0, 2 * z}, {-2 * w, -4 * z, 2 * y}};
    double dr3[4][3] = {{2 * y, -2 * x, 0}, {2 * z, -2 * w, -4 * x}, {2 * w, 2 * z, -4 * y}, {2 * x, 2 * y, 0}};
    double gh[4];
    for (int m = 0; m < 4; ++m) gh[m] = dot3(G1, dr1[m]) + dot3(G2, dr2[m]) + dot3(G3, dr3[m]);
    double proj = gh[0] * w + gh[1] * x + gh[2] * y + gh[3] * z;
    dq[0] = (gh[0] - proj * w) / qn;
    dq[1] = (gh[1] - proj * x) / qn;
    dq[2] = (gh[2] - proj * y) / qn;
    dq[3] = (gh[3] - proj * z) / qn;
}

/* Gradients of L with respect to every Gaussian parameter, given G = dL/d(spectrum) in
 * PyTorch's convention (dL/dRe + j dL/dIm), complex128 [n_lambda][H][W]:
 *   dL/dtheta = sum_f Re(conj(G(f)) d u_SLM(f) / dtheta).
 * blend 0: order-invariant sum.  blend 1: depth-sorted transmittance, including the
 * cross terms through T_i = prod (1 - alpha_j(mu_i)) (thresholded factors are held
 * fixed).  Outputs are per input index: dmean [n][3], dquat [n][4], dscale [n][2],
 * dopacity [n], damp [n][n_lambda]. */
void gwso_backward_spectrum(int64_t n, const double *mean, const double *quat, const double *scale,
                            const double *opacity, const double *amp, int n_lambda, const double *wavelengths,
                            int H, int W, double px, double py, int blend, int phase_match, double alpha_min,
                            const double *gspec, double *dmean, double *dquat, double *dscale, double *dopacity,
                            double *damp) {
    double *T = (double *)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    for (int64_t i = 0; i < n; ++i) T[i] = 1.0;
    if (blend == 1) gwso_transmittance(n, mean, quat, scale, opacity, alpha_min, T);
    /* dL/dw_il (w = c o T) */
    double *dw = (double *)calloc((size_t)(n > 0 ? n : 1) * n_lambda, sizeof(double));
    double *dR = (double *)calloc((size_t)(n > 0 ? n : 1) * 9, sizeof(double)); /* dL/dr1,r2,r3 */

#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t i = 0; i < n; ++i) {
        gauss_t G;
        load_gaussian(i, mean, quat, scale, opacity, &G);
        double dmu[3] = {0, 0, 0}, dsu = 0, dsv = 0, G1[3] = {0, 0, 0}, G2[3] = {0, 0, 0}, G3[3] = {0, 0, 0};
        for (int l = 0; l < n_lambda; ++l) {
            double wi = amp[i * n_lambda + l] * opacity[i] * T[i];
            double dwl = 0.0;
            for (int r = 0; r < H; ++r)
                for (int c = 0; c < W; ++c) {
                    freq_t f = grid_freq(r, c, H, W, px, py, wavelengths[l]);
                    if (!f.propagating) continue;
                    term_t t = gaussian_term(&G, &f, phase_match);
                    size_t o = ((size_t)l * H + r) * W + c;
                    double gr = gspec[2 * o], gi = gspec[2 * o + 1];
                    /* z = conj(G) * K  (K = unweighted term) */
                    double kr = gr * t.re + gi * t.im;
                    double ki = gr * t.im - gi * t.re;
                    dwl += kr;
                    double zr = wi * kr, zi = wi * ki;
                    double fv[3] = {f.fx, f.fy, f.fz};
                    double d[3] = {f.fx, f.fy, f.fz - f.inv_lam};
                    /* d/dmu: d u / d mu_k = -j 2 pi f_k u  ->  Re(conj(G)(-j)(...)) = Im(z) */
                    for (int k = 0; k < 3; ++k) dmu[k] += TWO_PI * fv[k] * zi;
                    if (phase_match) dmu[2] -= TWO_PI * f.inv_lam * zi;
                    dsu += zr * (1.0 / G.su - 4.0 * PI * PI * G.su * t.a * t.a);
                    dsv += zr * (1.0 / G.sv - 4.0 * PI * PI * G.sv * t.b * t.b);
                    for (int k = 0; k < 3; ++k) {
                        G1[k] += zr * (-4.0 * PI * PI * G.su * G.su * t.a) * d[k];
                        G2[k] += zr * (-4.0 * PI * PI * G.sv * G.sv * t.b) * d[k];
                        if (t.g != 0.0) G3[k] += zr * fv[k] / t.g;
                    }
                }
            dw[i * n_lambda + l] = dwl;
        }
        for (int k = 0; k < 3; ++k) {
            dmean[3 * i + k] = dmu[k];
            dR[9 * i + k] = G1[k];
            dR[9 * i + 3 + k] = G2[k];
            dR[9 * i + 6 + k] = G3[k];
        }
        dscale[2 * i] = dsu;
        dscale[2 * i + 1] = dsv;
    }

    /* colour, opacity and (sorted mode) transmittance */
    double *dT = (double *)calloc((size_t)(n > 0 ? n : 1), sizeof(double));
    for (int64_t i = 0; i < n; ++i) {
        double dopa = 0.0;
        for (int l = 0; l < n_lambda; ++l) {
            damp[i * n_lambda + l] = opacity[i] * T[i] * dw[i * n_lambda + l];
            dopa += amp[i * n_lambda + l] * T[i] * dw[i * n_lambda + l];
            dT[i] += amp[i * n_lambda + l] * opacity[i] * dw[i * n_lambda + l];
        }
        dopacity[i] = dopa;
    }
    if (blend == 1 && n > 0) {
        /* T_i = prod_{j in F_i} (1 - alpha_j(mu_i));  dT_i / d alpha_j = -prod_{k in F_i, k != j} (1 - alpha_k) */
        int64_t *order = (int64_t *)malloc(sizeof(int64_t) * (size_t)n);
        gwso_depth_order(n, mean, order);
        gauss_t *gs = (gauss_t *)malloc(sizeof(gauss_t) * (size_t)n);
        for (int64_t p = 0; p < n; ++p) load_gaussian(order[p], mean, quat, scale, opacity, &gs[p]);
        double *extra_mu = (double *)calloc((size_t)n * 3, sizeof(double));
        double *extra_s = (double *)calloc((size_t)n * 2, sizeof(double));
        double *extra_o = (double *)calloc((size_t)n, sizeof(double));
        double *extra_R = (double *)calloc((size_t)n * 6, sizeof(double)); /* dL/dr1_xy, dL/dr2_xy */
        double *alph = (double *)malloc(sizeof(double) * (size_t)n);
        /* sequential over (p, q): plain and deterministic */
        for (int64_t p = 0; p < n; ++p) {
            int64_t i = order[p];
            if (dT[i] == 0.0) continue;
            for (int64_t q = 0; q < p; ++q) alph[q] = alpha_at(&gs[q], gs[p].mu[0], gs[p].mu[1]);
            for (int64_t q = 0; q < p; ++q) {
                if (alph[q] < alpha_min) continue;
                double others = 1.0;
                for (int64_t k = 0; k < p; ++k)
                    if (k != q && alph[k] >= alpha_min) others *= (1.0 - alph[k]);
                double dA = -dT[i] * others; /* dL/d alpha_j(mu_i) */
                const gauss_t *g = &gs[q];
                int64_t j = order[q];
                double m00 = g->su * g->r1[0], m01 = g->sv * g->r2[0];
                double m10 = g->su * g->r1[1], m11 = g->sv * g->r2[1];
                double det = m00 * m11 - m01 * m10;
                double dx = gs[p].mu[0] - g->mu[0], dy = gs[p].mu[1] - g->mu[1];
                double y0 = (m11 * dx - m01 * dy) / det;
                double y1 = (-m10 * dx + m00 * dy) / det;
                double a = alph[q];
                /* alpha = o exp(-Q/2), Q = |y|^2, y = M^-1 d */
                extra_o[j] += dA * a / g->o;
                double dQ = dA * (-0.5 * a);
                /* dQ/dd = 2 M^-T y */
                double mty0 = (m11 * y0 - m10 * y1) / det;
                double mty1 = (-m01 * y0 + m00 * y1) / det;
                double gdx = dQ * 2.0 * mty0, gdy = dQ * 2.0 * mty1;
                extra_mu[3 * j] -= gdx;
                extra_mu[3 * j + 1] -= gdy;
                extra_mu[3 * i] += gdx;
                extra_mu[3 * i + 1] += gdy;
                /* dQ/dM = -2 (M^-T y) y^T ; M = [[su r1x, sv r2x], [su r1y, sv r2y]] */
                double gM00 = dQ * -2.0 * mty0 * y0, gM01 = dQ * -2.0 * mty0 * y1;
                double gM10 = dQ * -2.0 * mty1 * y0, gM11 = dQ * -2.0 * mty1 * y1;
                extra_s[2 * j] += gM00 * g->r1[0] + gM10 * g->r1[1];
                extra_s[2 * j + 1] += gM01 * g->r2[0] + gM11 * g->r2[1];
                extra_R[6 * j + 0] += gM00 * g->su;
                extra_R[6 * j + 1] += gM10 * g->su;
                extra_R[6 * j + 3] += gM01 * g->sv;
                extra_R[6 * j + 4] += gM11 * g->sv;
            }
        }
        for (int64_t i = 0; i < n; ++i) {
            dmean[3 * i] += extra_mu[3 * i];
            dmean[3 * i + 1] += extra_mu[3 * i + 1];
            dscale[2 * i] += extra_s[2 * i];
            dscale[2 * i + 1] += extra_s[2 * i + 1];
            dopacity[i] += extra_o[i];
            dR[9 * i + 0] += extra_R[6 * i + 0];
            dR[9 * i + 1] += extra_R[6 * i + 1];
            dR[9 * i + 3] += extra_R[6 * i + 3];
            dR[9 * i + 4] += extra_R[6 * i + 4];
        }
        free(alph);
        free(extra_R);
        free(extra_o);
        free(extra_s);
        free(extra_mu);
        free(gs);
        free(order);
    }
    for (int64_t i = 0; i < n; ++i) {
        gauss_t G;
        load_gaussian(i, mean, quat, scale, opacity, &G);
        quat_chain(G.qhat, G.qnorm, dR + 9 * i, dR + 9 * i + 3, dR + 9 * i + 6, dquat + 4 * i);
    }
    free(dT);
    free(dR);
    free(dw);
    free(T);
}

/* Order-invariant gradients (Eq. 12) of a subset of Gaussians only: for each input index in
 * `which`, the same per-Gaussian sums as gwso_backward_spectrum (every frequency of every
 * wavelength), O(H W L) per Gaussian.  Outputs are per entry of `which`. */
void gwso_backward_spectrum_at(int64_t n, const double *mean, const double *quat, const double *scale,
                               const double *opacity, const double *amp, int n_lambda, const double *wavelengths,
                               int H, int W, double px, double py, int phase_match, const double *gspec,
                               int64_t n_which, const int64_t *which, double *dmean, double *dquat, double *dscale,
                               double *dopacity, double *damp) {
    (void)n;
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t q = 0; q < n_which; ++q) {
        const int64_t i = which[q];
        gauss_t G;
        load_gaussian(i, mean, quat, scale, opacity, &G);
        double dmu[3] = {0, 0, 0}, dsu = 0, dsv = 0, G1[3] = {0, 0, 0}, G2[3] = {0, 0, 0}, G3[3] = {0, 0, 0};
        double dopa = 0.0;
        for (int l = 0; l < n_lambda; ++l) {
            double wi = amp[i * n_lambda + l] * opacity[i];
            double dwl = 0.0;
            for (int r = 0; r < H; ++r)
                for (int c = 0; c < W; ++c) {
                    freq_t f = grid_freq(r, c, H, W, px, py, wavelengths[l]);
                    if (!f.propagating) continue;
                    term_t t = gaussian_term(&G, &f, phase_match);
                    size_t o = ((size_t)l * H + r) * W + c;
                    double gr = gspec[2 * o], gi = gspec[2 * o + 1];
                    double kr = gr * t.re + gi * t.im;
                    double ki = gr * t.im - gi * t.re;
                    dwl += kr;
                    double zr = wi * kr, zi = wi * ki;
                    double fv[3] = {f.fx, f.fy, f.fz};
                    double d[3] = {f.fx, f.fy, f.fz - f.inv_lam};
                    for (int k = 0; k < 3; ++k) dmu[k] += TWO_PI * fv[k] * zi;
                    if (phase_match) dmu[2] -= TWO_PI * f.inv_lam * zi;
                    dsu += zr * (1.0 / G.su - 4.0 * PI * PI * G.su * t.a * t.a);
                    dsv += zr * (1.0 / G.sv - 4.0 * PI * PI * G.sv * t.b * t.b);
                    for (int k = 0; k < 3; ++k) {
                        G1[k] += zr * (-4.0 * PI * PI * G.su * G.su * t.a) * d[k];
                        G2[k] += zr * (-4.0 * PI * PI * G.sv * G.sv * t.b) * d[k];
                        if (t.g != 0.0) G3[k] += zr * fv[k] / t.g;
                    }
                }
            damp[q * n_lambda + l] = opacity[i] * dwl;
            dopa += amp[i * n_lambda + l] * dwl;
        }
        for (int k = 0; k < 3; ++k) dmean[3 * q + k] = dmu[k];
        dscale[2 * q] = dsu;
        dscale[2 * q + 1] = dsv;
        dopacity[q] = dopa;
        quat_chain(G.qhat, G.qnorm, G1, G2, G3, dquat + 4 * q);
    }
}

/* ------------------------------------------------------------------------------------ */
/* Exact alpha wave blending (Eq. 5-6 with the spatial transmittance map; Algorithm S2)  */
/* ------------------------------------------------------------------------------------ */

/* Front to back: for Gaussian k, u_k = the Gaussian's field on its own depth plane (Eq. 10
 * with the depth component of the mean set to zero, then the centred inverse DFT); the
 * SLM spectrum gains c_k o_k F(T u_k) H(f, -z_k) (F = the centred forward DFT scaled by
 * px py, the continuous transform on the grid); alpha_k = o_k |u_k|, kept where
 * alpha_k > t_eps (binarize > 0: alpha_k = 1 where alpha_k > binarize, else 0); then
 * T <- T (1 - alpha_k).  T starts at 1.  Writes the SLM spectrum (complex128
 * [n_lambda][H][W]) and, if T_out is not NULL, the final transmittance map [n_lambda][H][W]. */
void gwso_exact_awb(int64_t n, const double *mean, const double *quat, const double *scale, const double *opacity,
                    const double *amp, int n_lambda, const double *wavelengths, int H, int W, double px, double py,
                    double t_eps, double binarize, double *spec_out, double *T_out) {
    int64_t *order = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
    gwso_depth_order(n, mean, order);
    const size_t hw = (size_t)H * W;
    double *uhat = (double *)malloc(sizeof(double) * 2 * hw);
    double *u = (double *)malloc(sizeof(double) * 2 * hw);
    double *V = (double *)malloc(sizeof(double) * 2 * hw);
    double *T = (double *)malloc(sizeof(double) * hw);
    double dfx = 1.0 / (W * px), dfy = 1.0 / (H * py);
    for (int l = 0; l < n_lambda; ++l) {
        double *spec = spec_out + 2 * (size_t)l * hw;
        memset(spec, 0, sizeof(double) * 2 * hw);
        for (size_t k = 0; k < hw; ++k) T[k] = 1.0;
        for (int64_t p = 0; p < n; ++p) {
            int64_t i = order[p];
            gauss_t G;
            load_gaussian(i, mean, quat, scale, opacity, &G);
            const double zk = G.mu[2];
            G.mu[2] = 0.0; /* the field on the Gaussian's own plane */
            for (int r = 0; r < H; ++r)
                for (int c = 0; c < W; ++c) {
                    freq_t f = grid_freq(r, c, H, W, px, py, wavelengths[l]);
                    term_t t = gaussian_term(&G, &f, 0);
                    uhat[2 * ((size_t)r * W + c)] = t.re;
                    uhat[2 * ((size_t)r * W + c) + 1] = t.im;
                }
            centred_dft2(uhat, u, H, W, +1, dfx * dfy);
            const double co = amp[i * n_lambda + l] * opacity[i];
            for (size_t k = 0; k < hw; ++k) {
                V[2 * k] = co * T[k] * u[2 * k];
                V[2 * k + 1] = co * T[k] * u[2 * k + 1];
            }
            centred_dft2(V, uhat, H, W, -1, px * py); /* uhat <- F(c o T u_k) */
            for (int r = 0; r < H; ++r)
                for (int c = 0; c < W; ++c) {
                    freq_t f = grid_freq(r, c, H, W, px, py, wavelengths[l]);
                    if (!f.propagating) continue;
                    double cyc = -f.fz * zk; /* H(f, -z_k) = exp(-j 2 pi f_z z_k) */
                    cyc -= nearbyint(cyc);
                    const double cr = cos(TWO_PI * cyc), ci = sin(TWO_PI * cyc);
                    const size_t o = (size_t)r * W + c;
                    const double vr = uhat[2 * o], vi = uhat[2 * o + 1];
                    spec[2 * o] += vr * cr - vi * ci;
                    spec[2 * o + 1] += vr * ci + vi * cr;
                }
            for (size_t k = 0; k < hw; ++k) {
                double a = opacity[i] * hypot(u[2 * k], u[2 * k + 1]);
                if (!(a > t_eps)) a = 0.0;
                if (binarize > 0.0) a = (a > binarize) ? 1.0 : 0.0;
                T[k] *= (1.0 - a);
            }
        }
        if (T_out) memcpy(T_out + (size_t)l * hw, T, sizeof(double) * hw);
    }
    free(T);
    free(V);
    free(u);
    free(uhat);
    free(order);
}

int gwso_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void gwso_set_num_threads(int k) {
#ifdef _OPENMP
    if (k > 0) omp_set_num_threads(k);
#else
    (void)k;
#endif
}
