// gws_front.cu -- the holographics front end (Supplement Sec. 1.1: model, view, projective and
// hologram transforms with the 2D -> 3D lifting) and the view-dependent opacity of Sec. 4.2
// (alpha = G * SH(o, d)); one thread per Gaussian, FP64.
//
// With A_xy = Q R_q the thin QR of the hologram transform's first two columns (host, once per
// call) and C = R_q J W R_w diag(s) the 2x3 factor formed per Gaussian,
//   Sigma = A [[J W Sigma_w W^T J^T, 0], [0, 0]] A^T = A_xy (J W Sigma_w W^T J^T) A_xy^T = Q (C C^T) Q^T,
// so the eigendecomposition of the projected 2D covariance, the lifting and the factorisation
// Sigma = R S S^T R^T collapse into one closed-form eigendecomposition of the 2x2 P = C C^T:
// s_u^2 >= s_v^2 are its eigenvalues (det P = |c0 x c1|^2, free of cancellation) and
// r1, r2 = Q times its eigenvectors (taken algebraically: no FP64 transcendentals); r3 = r1 x r2
// is the normal of A's xy plane.
#include <math.h>

#include <cmath>

#include "gws_prep.h"

namespace gws {

struct FrontArgs {
    double W[9], t[3];      // view, row-major
    double fx, fy, cx, cy, z_near;
    double Q[6];            // 3x2, row-major [i][k]: orthonormal columns spanning A's xy block
    double r00, r01, r11;   // R_q
    double A[9], b[3];      // hologram transform, row-major
    double cam[3];          // camera centre -W^T t
    int proj, sh_degree, sh_stride;
};

// Real spherical harmonics of degree <= 3 at the unit direction d (Condon-Shortley phase,
// m = -l..l, normalised over the sphere), dotted with the coefficients c.
__device__ double sh_eval(const float *__restrict__ c, int degree, double x, double y, double z) {
    const double pi = 3.14159265358979323846;
    double v = c[0] * (0.5 / sqrt(pi));
    if (degree >= 1) {
        const double k1 = sqrt(3.0 / (4.0 * pi));
        v += k1 * (-(double)c[1] * y + (double)c[2] * z - (double)c[3] * x);
    }
    if (degree >= 2) {
        const double k2a = sqrt(15.0 / (4.0 * pi)), k2b = sqrt(5.0 / (16.0 * pi)), k2c = sqrt(15.0 / (16.0 * pi));
        v += k2a * ((double)c[4] * x * y - (double)c[5] * y * z - (double)c[7] * x * z) +
             k2b * (double)c[6] * (3.0 * z * z - 1.0) + k2c * (double)c[8] * (x * x - y * y);
    }
    if (degree >= 3) {
        const double k3a = sqrt(35.0 / (32.0 * pi)), k3b = sqrt(105.0 / (4.0 * pi)), k3c = sqrt(21.0 / (32.0 * pi));
        const double k3d = sqrt(7.0 / (16.0 * pi)), k3e = sqrt(105.0 / (16.0 * pi));
        const double z5 = 5.0 * z * z;
        v += -k3a * (double)c[9] * y * (3.0 * x * x - y * y) + k3b * (double)c[10] * x * y * z -
             k3c * (double)c[11] * y * (z5 - 1.0) + k3d * (double)c[12] * z * (z5 - 3.0) -
             k3c * (double)c[13] * x * (z5 - 1.0) + k3e * (double)c[14] * z * (x * x - y * y) -
             k3a * (double)c[15] * x * (x * x - 3.0 * y * y);
    }
    return v;
}

// Unit quaternion (w, x, y, z), w >= 0, of the rotation with columns r1, r2, r3 (Shepperd's
// method: the branch on the largest of the trace and the diagonal keeps the divisor >= 1).
__device__ void rot_to_quat(const double r1[3], const double r2[3], const double r3[3], double q[4]) {
    // R_ij: row i, column j; column j is r_{j+1}
    const double R00 = r1[0], R10 = r1[1], R20 = r1[2];
    const double R01 = r2[0], R11 = r2[1], R21 = r2[2];
    const double R02 = r3[0], R12 = r3[1], R22 = r3[2];
    const double tr = R00 + R11 + R22;
    double w, x, y, z;
    if (tr > 0.0) {
        const double S = 2.0 * sqrt(tr + 1.0);
        w = 0.25 * S;
        x = (R21 - R12) / S;
        y = (R02 - R20) / S;
        z = (R10 - R01) / S;
    } else if (R00 > R11 && R00 > R22) {
        const double S = 2.0 * sqrt(1.0 + R00 - R11 - R22);
        w = (R21 - R12) / S;
        x = 0.25 * S;
        y = (R01 + R10) / S;
        z = (R02 + R20) / S;
    } else if (R11 > R22) {
        const double S = 2.0 * sqrt(1.0 + R11 - R00 - R22);
        w = (R02 - R20) / S;
        x = (R01 + R10) / S;
        y = 0.25 * S;
        z = (R12 + R21) / S;
    } else {
        const double S = 2.0 * sqrt(1.0 + R22 - R00 - R11);
        w = (R10 - R01) / S;
        x = (R02 + R20) / S;
        y = (R12 + R21) / S;
        z = 0.25 * S;
    }
    const double sg = w < 0.0 ? -1.0 : 1.0;
    const double nrm = sg / sqrt(w * w + x * x + y * y + z * z);
    q[0] = w * nrm;
    q[1] = x * nrm;
    q[2] = y * nrm;
    q[3] = z * nrm;
}

__global__ void k_holographics(const double *__restrict__ mean_w, const float *__restrict__ quat_w,
                               const float *__restrict__ scale_w, const float *__restrict__ sh,
                               const float *__restrict__ opac_in, long long n, const __grid_constant__ FrontArgs F,
                               double *__restrict__ mean, float *__restrict__ quat, float *__restrict__ scale,
                               float *__restrict__ opacity, unsigned char *__restrict__ valid) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double mw[3] = {mean_w[3 * i], mean_w[3 * i + 1], mean_w[3 * i + 2]};
    double qw[4] = {quat_w[4 * i], quat_w[4 * i + 1], quat_w[4 * i + 2], quat_w[4 * i + 3]};
    const double s[3] = {scale_w[3 * i], scale_w[3 * i + 1], scale_w[3 * i + 2]};
    const double qn = sqrt(qw[0] * qw[0] + qw[1] * qw[1] + qw[2] * qw[2] + qw[3] * qw[3]);
    bool ok = isfinite(mw[0]) && isfinite(mw[1]) && isfinite(mw[2]) && isfinite(qn) && qn > 0.0 && isfinite(s[0]) &&
              isfinite(s[1]) && isfinite(s[2]) && s[0] >= 0.0 && s[1] >= 0.0 && s[2] >= 0.0;
    // view transform
    double xv[3];
#pragma unroll
    for (int r = 0; r < 3; ++r) xv[r] = F.W[3 * r] * mw[0] + F.W[3 * r + 1] * mw[1] + F.W[3 * r + 2] * mw[2] + F.t[r];
    // in front: view depth -z at least z_near (and z < 0 where phi divides by -z)
    ok = ok && -xv[2] >= F.z_near && (F.proj != GWS_PROJ_PERSPECTIVE || xv[2] < 0.0);
    double out_mean[3] = {0.0, 0.0, 0.0}, out_q[4] = {1.0, 0.0, 0.0, 0.0}, su = 0.0, sv = 0.0, op = 0.0;
    if (ok) {
        // projective mapping and its Jacobian J = [[j00, 0, j02], [0, j11, j12]] at the mean
        double u, v, j00, j02, j11, j12;
        if (F.proj == GWS_PROJ_PERSPECTIVE) {
            const double iz = 1.0 / (-xv[2]);
            u = F.fx * xv[0] * iz + F.cx;
            v = F.fy * xv[1] * iz + F.cy;
            j00 = F.fx * iz;
            j11 = F.fy * iz;
            j02 = F.fx * xv[0] * iz * iz;
            j12 = F.fy * xv[1] * iz * iz;
        } else {
            u = F.fx * xv[0] + F.cx;
            v = F.fy * xv[1] + F.cy;
            j00 = F.fx;
            j11 = F.fy;
            j02 = j12 = 0.0;
        }
        // K = R_q J, then C = K W R_w diag(s)
        const double K[2][3] = {{F.r00 * j00, F.r01 * j11, F.r00 * j02 + F.r01 * j12},
                                {0.0, F.r11 * j11, F.r11 * j12}};
        double KW[2][3];
#pragma unroll
        for (int a = 0; a < 2; ++a)
#pragma unroll
            for (int k = 0; k < 3; ++k) KW[a][k] = K[a][0] * F.W[k] + K[a][1] * F.W[3 + k] + K[a][2] * F.W[6 + k];
        const double qh[4] = {qw[0] / qn, qw[1] / qn, qw[2] / qn, qw[3] / qn};
        double r1w[3], r2w[3], r3w[3];
        quat_cols<double>(qh, r1w, r2w, r3w);
        double c[2][3];
#pragma unroll
        for (int a = 0; a < 2; ++a) {
            c[a][0] = (KW[a][0] * r1w[0] + KW[a][1] * r1w[1] + KW[a][2] * r1w[2]) * s[0];
            c[a][1] = (KW[a][0] * r2w[0] + KW[a][1] * r2w[1] + KW[a][2] * r2w[2]) * s[1];
            c[a][2] = (KW[a][0] * r3w[0] + KW[a][1] * r3w[1] + KW[a][2] * r3w[2]) * s[2];
        }
        // P = C C^T = V diag(s_u^2, s_v^2) V^T
        const double p00 = c[0][0] * c[0][0] + c[0][1] * c[0][1] + c[0][2] * c[0][2];
        const double p11 = c[1][0] * c[1][0] + c[1][1] * c[1][1] + c[1][2] * c[1][2];
        const double p01 = c[0][0] * c[1][0] + c[0][1] * c[1][1] + c[0][2] * c[1][2];
        const double x0 = c[0][1] * c[1][2] - c[0][2] * c[1][1];
        const double x1 = c[0][2] * c[1][0] - c[0][0] * c[1][2];
        const double x2 = c[0][0] * c[1][1] - c[0][1] * c[1][0];
        const double det = x0 * x0 + x1 * x1 + x2 * x2;
        const double half = 0.5 * (p00 - p11);
        const double h = sqrt(half * half + p01 * p01);
        const double lam1 = 0.5 * (p00 + p11) + h;
        const double lam2 = lam1 > 0.0 ? det / lam1 : 0.0;
        // eigenvector of lam1 from the row of P - lam1 I with the larger norm: (h + half, p01)
        // or (p01, h - half); any unit vector when P is isotropic
        double e0 = half >= 0.0 ? h + half : p01, e1 = half >= 0.0 ? p01 : h - half;
        const double en = e0 * e0 + e1 * e1;
        double cs = 1.0, sn = 0.0;
        if (en > 0.0) {
            const double ie = 1.0 / sqrt(en);
            cs = e0 * ie;
            sn = e1 * ie;
        }
        double r1[3], r2[3], r3[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            r1[k] = F.Q[2 * k] * cs + F.Q[2 * k + 1] * sn;
            r2[k] = -F.Q[2 * k] * sn + F.Q[2 * k + 1] * cs;
        }
        r3[0] = r1[1] * r2[2] - r1[2] * r2[1];
        r3[1] = r1[2] * r2[0] - r1[0] * r2[2];
        r3[2] = r1[0] * r2[1] - r1[1] * r2[0];
        rot_to_quat(r1, r2, r3, out_q);
        su = sqrt(lam1);
        sv = sqrt(lam2);
        // mu = A (u, v, z_view) + b
        const double mv[3] = {u, v, xv[2]};
#pragma unroll
        for (int r = 0; r < 3; ++r) out_mean[r] = F.A[3 * r] * mv[0] + F.A[3 * r + 1] * mv[1] + F.A[3 * r + 2] * mv[2] + F.b[r];
        // opacity: SH(o, d), d = unit(mu_w - camera centre), clamped to [0, 1]
        if (sh) {
            const double d0 = mw[0] - F.cam[0], d1 = mw[1] - F.cam[1], d2 = mw[2] - F.cam[2];
            const double idn = 1.0 / sqrt(d0 * d0 + d1 * d1 + d2 * d2);
            op = sh_eval(sh + (size_t)i * F.sh_stride, F.sh_degree, d0 * idn, d1 * idn, d2 * idn);
            op = fmin(fmax(op, 0.0), 1.0);
        } else {
            op = opac_in[i];
        }
        // a footprint of zero area carries no weight (W ~ s_u s_v): culled like a hidden one
        ok = (float)su > 0.f && (float)sv > 0.f && isfinite(op) && isfinite(out_mean[0]) && isfinite(out_mean[1]) &&
             isfinite(out_mean[2]);
        if (!ok) {
            out_mean[0] = out_mean[1] = out_mean[2] = 0.0;
            out_q[0] = 1.0;
            out_q[1] = out_q[2] = out_q[3] = 0.0;
            su = sv = op = 0.0;
        }
    }
    mean[3 * i] = out_mean[0];
    mean[3 * i + 1] = out_mean[1];
    mean[3 * i + 2] = out_mean[2];
#pragma unroll
    for (int k = 0; k < 4; ++k) quat[4 * i + k] = (float)out_q[k];
    scale[2 * i] = (float)su;
    scale[2 * i + 1] = (float)sv;
    opacity[i] = (float)op;
    if (valid) valid[i] = ok ? 1 : 0;
}

}  // namespace gws

extern "C" gws_status gws_holographics(const gws_world_gaussians *in, int64_t n, const gws_camera *cam,
                                       const double holo[12], const gws_opts *opts, gws_gaussians_out *out,
                                       unsigned char *valid) {
    using namespace gws;
    if (!in || !cam || !holo || !opts || !out || n < 0) return GWS_ERR_INVALID_ARG;
    if (in->sh_degree < 0 || in->sh_degree > 3) return GWS_ERR_INVALID_ARG;
    const int K = (in->sh_degree + 1) * (in->sh_degree + 1);
    const int stride = in->sh_stride == 0 ? K : in->sh_stride;
    if (stride < K) return GWS_ERR_INVALID_ARG;
    if (cam->projection != GWS_PROJ_PERSPECTIVE && cam->projection != GWS_PROJ_ORTHOGRAPHIC) return GWS_ERR_INVALID_ARG;
    FrontArgs F;
    for (int k = 0; k < 12; ++k)
        if (!std::isfinite(cam->view[k]) || !std::isfinite(holo[k])) return GWS_ERR_INVALID_ARG;
    if (!std::isfinite(cam->fx) || !std::isfinite(cam->fy) || !std::isfinite(cam->cx) || !std::isfinite(cam->cy) ||
        !std::isfinite(cam->z_near))
        return GWS_ERR_INVALID_ARG;
    for (int r = 0; r < 3; ++r) {
        for (int k = 0; k < 3; ++k) {
            F.W[3 * r + k] = cam->view[4 * r + k];
            F.A[3 * r + k] = holo[4 * r + k];
        }
        F.t[r] = cam->view[4 * r + 3];
        F.b[r] = holo[4 * r + 3];
    }
    for (int k = 0; k < 3; ++k) F.cam[k] = -(F.W[k] * F.t[0] + F.W[3 + k] * F.t[1] + F.W[6 + k] * F.t[2]);
    // thin QR of A's first two columns (Gram-Schmidt, applied twice for orthogonality)
    const double a1[3] = {F.A[0], F.A[3], F.A[6]}, a2[3] = {F.A[1], F.A[4], F.A[7]};
    const double n1 = std::sqrt(a1[0] * a1[0] + a1[1] * a1[1] + a1[2] * a1[2]);
    const double n2 = std::sqrt(a2[0] * a2[0] + a2[1] * a2[1] + a2[2] * a2[2]);
    if (!(n1 > 0.0) || !(n2 > 0.0)) return GWS_ERR_INVALID_ARG;
    double q1[3], u[3];
    for (int k = 0; k < 3; ++k) q1[k] = a1[k] / n1;
    double r01 = q1[0] * a2[0] + q1[1] * a2[1] + q1[2] * a2[2];
    for (int k = 0; k < 3; ++k) u[k] = a2[k] - r01 * q1[k];
    const double c2 = q1[0] * u[0] + q1[1] * u[1] + q1[2] * u[2];
    r01 += c2;
    for (int k = 0; k < 3; ++k) u[k] -= c2 * q1[k];
    const double r11 = std::sqrt(u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
    if (!(r11 > 1e-12 * n2)) return GWS_ERR_INVALID_ARG;  // A's xy columns (nearly) parallel
    for (int k = 0; k < 3; ++k) {
        F.Q[2 * k] = q1[k];
        F.Q[2 * k + 1] = u[k] / r11;
    }
    F.r00 = n1;
    F.r01 = r01;
    F.r11 = r11;
    F.fx = cam->fx;
    F.fy = cam->fy;
    F.cx = cam->cx;
    F.cy = cam->cy;
    F.z_near = cam->z_near;
    F.proj = cam->projection;
    F.sh_degree = in->sh_degree;
    F.sh_stride = stride;
    if (n == 0) return GWS_OK;
    if (!in->mean || !in->quat || !in->scale || (!in->sh_opacity && !in->opacity)) return GWS_ERR_INVALID_ARG;
    if (!out->mean || !out->quat || !out->scale || !out->opacity) return GWS_ERR_INVALID_ARG;
    k_holographics<<<(unsigned)((n + 127) / 128), 128, 0, (cudaStream_t)opts->stream>>>(
        in->mean, in->quat, in->scale, in->sh_opacity, in->opacity, (long long)n, F, out->mean, out->quat, out->scale,
        out->opacity, valid);
    count_launches(1);
    return cudaGetLastError() == cudaSuccess ? GWS_OK : GWS_ERR_CUDA;
}
