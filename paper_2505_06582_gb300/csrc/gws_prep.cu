// gws_prep.cu -- everything on the hot path except the splats:
//   validation + per-Gaussian precompute, depth keys (Algorithm S2 order), the
//   transmittance at each centre (Eq. 2, Eq. 5-6 reading, t_eps of Algorithm S2), FP64
//   records, spectral footprints + footprint-ordered records (binning), work items,
//   centred-DFT modulations around cuFFT (Eq. 3 on the grid) and double-phase encoding.
#include <float.h>

#include <algorithm>

#include "gws_prep.h"

namespace gws {

// ---------------------------------------------------------------------------------------
// validation, normalised quaternion, depth key
// ---------------------------------------------------------------------------------------

__device__ __forceinline__ unsigned long long depth_key(double z) {
    z = z + 0.0;  // -0 == +0: equal depths tie (input order decides)
    unsigned long long b = (unsigned long long)__double_as_longlong(z);
    return (b & 0x8000000000000000ull) ? ~b : (b | 0x8000000000000000ull);
}

__global__ void k_prep(const __grid_constant__ SceneTable T, long long n_total, GPre *__restrict__ gp,
                       float *__restrict__ ampc, unsigned long long *__restrict__ dkey, unsigned *__restrict__ dval,
                       int *__restrict__ status) {
    const long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= n_total) return;
    const int s = scene_of(T.off, T.n_scenes, g);
    const long long i = g - T.off[s];
    const int L = T.n_lambda;
    double mu[3] = {T.mean[s][3 * i], T.mean[s][3 * i + 1], T.mean[s][3 * i + 2]};
    double q[4] = {T.quat[s][4 * i], T.quat[s][4 * i + 1], T.quat[s][4 * i + 2], T.quat[s][4 * i + 3]};
    float su = T.scale[s][2 * i], sv = T.scale[s][2 * i + 1], o = T.opacity[s][i];
    int bad = 0;
    bool fin = isfinite(mu[0]) && isfinite(mu[1]) && isfinite(mu[2]) && isfinite(q[0]) && isfinite(q[1]) &&
               isfinite(q[2]) && isfinite(q[3]) && isfinite(su) && isfinite(sv) && isfinite(o);
    for (int l = 0; l < L; ++l) {
        float c = T.amp[s][i * L + l];
        fin = fin && isfinite(c);
        ampc[g * L + l] = c;
    }
    const double qn = sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
    if (!fin) bad |= ST_NONFINITE;
    else if (!(su > 0.f) || !(sv > 0.f) || !(o >= 0.f && o <= 1.f) || !(qn > 0.0)) bad |= ST_BADVALUE;
    if (bad) {
        atomicOr(status, bad);
        if (!(qn > 0.0) || !isfinite(qn)) {
            q[0] = 1.0;
            q[1] = q[2] = q[3] = 0.0;
        }
    }
    GPre r;
    r.mu[0] = mu[0];
    r.mu[1] = mu[1];
    r.mu[2] = mu[2];
    const double inv = (qn > 0.0 && isfinite(qn)) ? 1.0 / qn : 1.0;
    for (int k = 0; k < 4; ++k) r.q[k] = (qn > 0.0 && isfinite(qn)) ? q[k] / qn : q[k] * inv;
    r.su = su;
    r.sv = sv;
    r.o = o;
    r.scene = s;
    gp[g] = r;
    dkey[g] = depth_key(mu[2]);
    dval[g] = (unsigned)g;
}

// scene id of each depth-sorted entry, for the final (stable) grouping pass
__global__ void k_scene_key(const GPre *__restrict__ gp, const unsigned *__restrict__ sorted, long long n,
                            unsigned *__restrict__ skey) {
    const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (p < n) skey[p] = (unsigned)gp[sorted[p]].scene;
}

// ---------------------------------------------------------------------------------------
// transmittance at the centres (depth-sorted)
// ---------------------------------------------------------------------------------------

__global__ void k_tdata(const GPre *__restrict__ gp, const unsigned *__restrict__ sorted, long long n,
                        double alpha_min, TData *__restrict__ td) {
    const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    const GPre &g = gp[sorted[p]];
    double r1[3], r2[3], r3[3];
    quat_cols<double>(g.q, r1, r2, r3);
    TData t;
    t.mx = g.mu[0];
    t.my = g.mu[1];
    t.m00 = (double)g.su * r1[0];
    t.m01 = (double)g.sv * r2[0];
    t.m10 = (double)g.su * r1[1];
    t.m11 = (double)g.sv * r2[1];
    t.det = t.m00 * t.m11 - t.m01 * t.m10;
    t.o = g.o;
    t.pad = 0.f;
    const bool edge_on = fabs(t.det) < 1e-14 * (double)g.su * (double)g.sv;
    if (edge_on || !((double)g.o >= alpha_min) || g.o <= 0.f) {
        t.bx0 = 1.f;
        t.bx1 = -1.f;
        t.by0 = 1.f;
        t.by1 = -1.f;
    } else {
        // alpha >= alpha_min  <=>  |M^-1 d|^2 <= 2 ln(o / alpha_min); box of that ellipse
        const double qmax = 2.0 * log((double)g.o / alpha_min);
        const double hx = sqrt(fmax(qmax, 0.0) * (t.m00 * t.m00 + t.m01 * t.m01)) * 1.0001 + 1e-12;
        const double hy = sqrt(fmax(qmax, 0.0) * (t.m10 * t.m10 + t.m11 * t.m11)) * 1.0001 + 1e-12;
        t.bx0 = __double2float_rd(t.mx - hx);
        t.bx1 = __double2float_ru(t.mx + hx);
        t.by0 = __double2float_rd(t.my - hy);
        t.by1 = __double2float_ru(t.my + hy);
    }
    td[p] = t;
}

constexpr int kTChunk = 128;

// T_p = prod over earlier (front) entries q of the same scene of (1 - alpha_q(mu_p)),
// alpha below alpha_min dropped.  FP64 like the oracle; boxes cull in FP32 (conservative).
__global__ void __launch_bounds__(kTChunk) k_transmit(const TData *__restrict__ td, const unsigned *__restrict__ sorted,
                                                      Segs S, long long n, double alpha_min,
                                                      double *__restrict__ T_sorted, double *__restrict__ T_g,
                                                      TQuery *__restrict__ tq) {
    __shared__ TData s_td[kTChunk];
    const long long p = (long long)blockIdx.x * kTChunk + threadIdx.x;
    const bool active = p < n;
    const long long pp = active ? p : n - 1;
    const int sc = scene_of(S.off, S.n_scenes, pp);
    const long long start = S.off[sc];
    const double xp = td[pp].mx, yp = td[pp].my;
    const float xf = (float)xp, yf = (float)yp;
    // block range of fronts: [min start in block, max p in block)
    const long long pfirst = (long long)blockIdx.x * kTChunk;
    const long long plast = min(pfirst + kTChunk, n) - 1;
    const long long qlo = S.off[scene_of(S.off, S.n_scenes, pfirst)];
    double T = 1.0, Tnz = 1.0;
    int n1 = 0;
    for (long long c0 = qlo; c0 < plast; c0 += kTChunk) {
        __syncthreads();
        if (c0 + threadIdx.x < plast) s_td[threadIdx.x] = td[c0 + threadIdx.x];
        __syncthreads();
        const long long cend = min((long long)kTChunk, plast - c0);
        for (int k = 0; k < cend; ++k) {
            const long long q = c0 + k;
            if (q < start || q >= pp) continue;
            const TData &f = s_td[k];
            if (xf < f.bx0 || xf > f.bx1 || yf < f.by0 || yf > f.by1) continue;
            const double dx = xp - f.mx, dy = yp - f.my;
            const double y0 = (f.m11 * dx - f.m01 * dy) / f.det;
            const double y1 = (-f.m10 * dx + f.m00 * dy) / f.det;
            const double a = (double)f.o * exp(-0.5 * (y0 * y0 + y1 * y1));
            if (a >= alpha_min) {
                T *= (1.0 - a);
                if (a == 1.0) ++n1;
                else Tnz *= (1.0 - a);
            }
        }
    }
    if (active) {
        T_sorted[p] = T;
        T_g[sorted[p]] = T;
        if (tq) {
            TQuery q;
            q.Tnz = Tnz;
            q.dT = 0.0;
            q.n1 = n1;
            q.pad = 0;
            tq[p] = q;
        }
    }
}

// ---------------------------------------------------------------------------------------
// backward cross terms through the transmittance (depth-sorted mode)
//   T_i = prod_{j front of i, alpha_j(mu_i) >= alpha_min} (1 - alpha_j(mu_i)),
//   alpha_j(x) = o_j exp(-Q/2),  Q = |M_j^-1 (x - mu_j)_xy|^2,  M_j = [s_u r1_xy, s_v r2_xy];
//   dL/dalpha_j(mu_i) = -dL/dT_i prod_{k != j} (1 - alpha_k(mu_i))  (the threshold set held fixed)
// ---------------------------------------------------------------------------------------

__device__ __forceinline__ double others_product(const TQuery &q, double a) {
    if (q.n1 == 0) return q.Tnz / (1.0 - a);
    if (q.n1 == 1 && a == 1.0) return q.Tnz;
    return 0.0;
}

__global__ void k_tq_dT(const unsigned *__restrict__ sorted, const double *__restrict__ dT_g, long long n,
                        TQuery *__restrict__ tq) {
    const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (p < n) tq[p].dT = dT_g[sorted[p]];
}

// pass A: per Gaussian i (sorted position p), the terms on its own mean (d = mu_i - mu_j)
__global__ void __launch_bounds__(kTChunk) k_tgrad_query(const TData *__restrict__ td, const TQuery *__restrict__ tq,
                                                         const unsigned *__restrict__ sorted, Segs S, long long n,
                                                         double alpha_min, double *__restrict__ dmean) {
    __shared__ TData s_td[kTChunk];
    const long long p = (long long)blockIdx.x * kTChunk + threadIdx.x;
    const bool active = p < n;
    const long long pp = active ? p : n - 1;
    const long long start = S.off[scene_of(S.off, S.n_scenes, pp)];
    const double xp = td[pp].mx, yp = td[pp].my;
    const float xf = (float)xp, yf = (float)yp;
    const TQuery Q = tq[pp];
    const long long pfirst = (long long)blockIdx.x * kTChunk;
    const long long plast = min(pfirst + kTChunk, n) - 1;
    const long long qlo = S.off[scene_of(S.off, S.n_scenes, pfirst)];
    double gx = 0.0, gy = 0.0;
    for (long long c0 = qlo; c0 < plast; c0 += kTChunk) {
        __syncthreads();
        if (c0 + threadIdx.x < plast) s_td[threadIdx.x] = td[c0 + threadIdx.x];
        __syncthreads();
        const long long cend = min((long long)kTChunk, plast - c0);
        if (Q.dT == 0.0) continue;
        for (int k = 0; k < cend; ++k) {
            const long long q = c0 + k;
            if (q < start || q >= pp) continue;
            const TData &f = s_td[k];
            if (xf < f.bx0 || xf > f.bx1 || yf < f.by0 || yf > f.by1) continue;
            const double dx = xp - f.mx, dy = yp - f.my;
            const double y0 = (f.m11 * dx - f.m01 * dy) / f.det;
            const double y1 = (-f.m10 * dx + f.m00 * dy) / f.det;
            const double a = (double)f.o * exp(-0.5 * (y0 * y0 + y1 * y1));
            if (a < alpha_min) continue;
            const double dA = -Q.dT * others_product(Q, a);
            const double dQ = dA * (-0.5 * a);
            const double mty0 = (f.m11 * y0 - f.m10 * y1) / f.det;
            const double mty1 = (-f.m01 * y0 + f.m00 * y1) / f.det;
            gx += dQ * 2.0 * mty0;
            gy += dQ * 2.0 * mty1;
        }
    }
    if (active) {
        const unsigned g = sorted[p];
        dmean[3 * (size_t)g] += gx;
        dmean[3 * (size_t)g + 1] += gy;
    }
}

// pass B: per front Gaussian j (sorted position q), the terms on its mean, scales, rotation
// and opacity, summed over the Gaussians i behind it
__global__ void __launch_bounds__(kTChunk) k_tgrad_front(const TData *__restrict__ td, const TQuery *__restrict__ tq,
                                                         const GPre *__restrict__ gp, const unsigned *__restrict__ sorted,
                                                         const float *__restrict__ quat_in, Segs S, long long n,
                                                         double alpha_min, double *__restrict__ dmean,
                                                         float *__restrict__ dquat, float *__restrict__ dscale,
                                                         float *__restrict__ dopacity) {
    __shared__ double s_x[kTChunk], s_y[kTChunk];
    __shared__ TQuery s_q[kTChunk];
    const long long q = (long long)blockIdx.x * kTChunk + threadIdx.x;
    const bool active = q < n;
    const long long qq = active ? q : n - 1;
    const int sc = scene_of(S.off, S.n_scenes, qq);
    const long long end = S.off[sc + 1];
    const TData f = td[qq];
    const long long qfirst = (long long)blockIdx.x * kTChunk;
    const long long plo = qfirst + 1;
    const long long phi = S.off[scene_of(S.off, S.n_scenes, min(qfirst + kTChunk, n) - 1) + 1];
    double go = 0.0, gmx = 0.0, gmy = 0.0, gM00 = 0.0, gM01 = 0.0, gM10 = 0.0, gM11 = 0.0;
    const bool has_box = !(f.bx0 > f.bx1);
    for (long long c0 = plo; c0 < phi; c0 += kTChunk) {
        __syncthreads();
        if (c0 + threadIdx.x < phi) {
            s_x[threadIdx.x] = td[c0 + threadIdx.x].mx;
            s_y[threadIdx.x] = td[c0 + threadIdx.x].my;
            s_q[threadIdx.x] = tq[c0 + threadIdx.x];
        }
        __syncthreads();
        if (!has_box) continue;
        const long long cend = min((long long)kTChunk, phi - c0);
        for (int k = 0; k < cend; ++k) {
            const long long p = c0 + k;
            if (p <= qq || p >= end) continue;
            const float xf = (float)s_x[k], yf = (float)s_y[k];
            if (xf < f.bx0 || xf > f.bx1 || yf < f.by0 || yf > f.by1) continue;
            const TQuery &Q = s_q[k];
            if (Q.dT == 0.0) continue;
            const double dx = s_x[k] - f.mx, dy = s_y[k] - f.my;
            const double y0 = (f.m11 * dx - f.m01 * dy) / f.det;
            const double y1 = (-f.m10 * dx + f.m00 * dy) / f.det;
            const double a = (double)f.o * exp(-0.5 * (y0 * y0 + y1 * y1));
            if (a < alpha_min) continue;
            const double dA = -Q.dT * others_product(Q, a);
            if (f.o > 0.f) go += dA * a / (double)f.o;
            const double dQ = dA * (-0.5 * a);
            const double mty0 = (f.m11 * y0 - f.m10 * y1) / f.det;
            const double mty1 = (-f.m01 * y0 + f.m00 * y1) / f.det;
            gmx -= dQ * 2.0 * mty0;
            gmy -= dQ * 2.0 * mty1;
            gM00 += dQ * -2.0 * mty0 * y0;
            gM01 += dQ * -2.0 * mty0 * y1;
            gM10 += dQ * -2.0 * mty1 * y0;
            gM11 += dQ * -2.0 * mty1 * y1;
        }
    }
    if (!active) return;
    const unsigned g = sorted[q];
    const GPre &P = gp[g];
    double r1[3], r2[3], r3[3];
    quat_cols<double>(P.q, r1, r2, r3);
    const double su = P.su, sv = P.sv;
    const double dsu = gM00 * r1[0] + gM10 * r1[1], dsv = gM01 * r2[0] + gM11 * r2[1];
    const double G1[3] = {gM00 * su, gM10 * su, 0.0}, G2[3] = {gM01 * sv, gM11 * sv, 0.0};
    const double w = P.q[0], x = P.q[1], y = P.q[2], z = P.q[3];
    const double dr1[4][3] = {{0, 2 * z, -2 * y}, {0, 2 * y, 2 * z}, {-4 * y, 2 * x, -2 * w}, {-4 * z, 2 * w, 2 * x}};
    const double dr2[4][3] = {{-2 * z, 0, 2 * x}, {2 * y, -4 * x, 2 * w}, {2 * x, 0, 2 * z}, {-2 * w, -4 * z, 2 * y}};
    double gh[4];
    for (int m = 0; m < 4; ++m) {
        gh[m] = 0;
        for (int k = 0; k < 3; ++k) gh[m] += G1[k] * dr1[m][k] + G2[k] * dr2[m][k];
    }
    const double qi[4] = {quat_in[4 * g], quat_in[4 * g + 1], quat_in[4 * g + 2], quat_in[4 * g + 3]};
    const double qn = sqrt(qi[0] * qi[0] + qi[1] * qi[1] + qi[2] * qi[2] + qi[3] * qi[3]);
    const double proj = gh[0] * w + gh[1] * x + gh[2] * y + gh[3] * z;
    const double qh[4] = {w, x, y, z};
    for (int m = 0; m < 4; ++m) dquat[4 * (size_t)g + m] = (float)((double)dquat[4 * (size_t)g + m] + (gh[m] - proj * qh[m]) / qn);
    dmean[3 * (size_t)g] += gmx;
    dmean[3 * (size_t)g + 1] += gmy;
    dscale[2 * (size_t)g] = (float)((double)dscale[2 * (size_t)g] + dsu);
    dscale[2 * (size_t)g + 1] = (float)((double)dscale[2 * (size_t)g + 1] + dsv);
    dopacity[g] = (float)((double)dopacity[g] + go);
}

// ---------------------------------------------------------------------------------------
// FP64 path records
// ---------------------------------------------------------------------------------------

__global__ void k_rec64(const GPre *__restrict__ gp, const float *__restrict__ ampc,
                        const unsigned *__restrict__ sorted, const double *__restrict__ T_sorted, long long n, int L,
                        Rec64 *__restrict__ rec, double *__restrict__ w) {
    const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    const unsigned g = sorted[p];
    const GPre &G = gp[g];
    Rec64 r;
    quat_cols<double>(G.q, r.r1, r.r2, r.r3);
    r.mu[0] = G.mu[0];
    r.mu[1] = G.mu[1];
    r.mu[2] = G.mu[2];
    r.su = G.su;
    r.sv = G.sv;
    rec[p] = r;
    const double T = T_sorted ? T_sorted[p] : 1.0;
    for (int l = 0; l < L; ++l) w[p * L + l] = (double)ampc[(size_t)g * L + l] * (double)G.o * T;
}

// ---------------------------------------------------------------------------------------
// spectral footprints and footprint-ordered records (the MIXED path's binning)
// ---------------------------------------------------------------------------------------

struct Foot {
    float e00, e01, e11, R;
    float wz;  // |(s_u r1z, s_v r2z)| / rho' (rho' before the 1.0005 margin)
};

// Frequencies with |M^T f| > rho' have E = 2 pi^2 (s_u^2 a^2 + s_v^2 b^2) > ln(1/eps): with
// v = (s_u a, s_v b) = M^T f + d_z (s_u r1z, s_v r2z) and |d_z| <= dzmax on the grid,
// |v| <= rho  implies  |M^T f| <= rho + dzmax |(s_u r1z, s_v r2z)| = rho'.
// The footprint is the ellipse f^T (M M^T / rho'^2) f <= 1, centred at f = 0 (the
// reference-wave shift puts every Gaussian's spectral peak at the origin).  R bounds its
// largest radius.
__device__ __forceinline__ Foot footprint(const float r1[3], const float r2[3], float su, float sv, float rho,
                                          float dzmax) {
    const float m00 = su * r1[0], m01 = sv * r2[0], m10 = su * r1[1], m11 = sv * r2[1];
    const float a00 = m00 * m00 + m01 * m01, a01 = m00 * m10 + m01 * m11, a11 = m10 * m10 + m11 * m11;
    const float cz = sqrtf(su * su * r1[2] * r1[2] + sv * sv * r2[2] * r2[2]);
    float rp = rho + dzmax * cz;
    const float wz = cz / rp;
    rp *= 1.0005f;
    const float inv = 1.f / (rp * rp);
    Foot f;
    f.e00 = a00 * inv;
    f.e01 = a01 * inv;
    f.e11 = a11 * inv;
    const float det = m00 * m11 - m01 * m10;
    const float det2 = det * det;
    const float half = 0.5f * (a00 + a11);
    const float disc = sqrtf(fmaxf(0.25f * (a00 - a11) * (a00 - a11) + a01 * a01, 0.f));
    const float lmax = half + disc;
    const float lmin = lmax > 0.f ? det2 / lmax : 0.f;
    f.R = (lmin > 1e-30f * lmax && lmin > 0.f) ? 1.002f * rp / sqrtf(lmin) : FLT_MAX;
    f.wz = wz;
    return f;
}

// Rotation columns formed in FP64 and rounded once: in FP32, 1 - 2 (x^2 + y^2) loses the small
// components (a near edge-on Gaussian's r3_z ~ 1e-5 came out ~5e-8 off, and the |r3.f| kink of
// Eq. 10 makes the gradient through r3 jump when that moves pixels across r3.f = 0).
__device__ __forceinline__ void cols_f32(const double qd[4], float r1[3], float r2[3], float r3[3]) {
    double d1[3], d2[3], d3[3];
    quat_cols<double>(qd, d1, d2, d3);
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        r1[k] = (float)d1[k];
        r2[k] = (float)d2[k];
        r3[k] = (float)d3[k];
    }
}

// record slot k (segment-major, depth order inside a segment) -> (segment, sorted position)
__device__ __forceinline__ void slot_decode(const Segs &S, long long k, int &seg, long long &p) {
    // find scene s with L off[s] <= k < L off[s+1]
    const int L = S.n_lambda;
    int lo = 0, hi = S.n_scenes - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if ((long long)L * S.off[mid] <= k) lo = mid;
        else hi = mid - 1;
    }
    const long long ns = S.off[lo + 1] - S.off[lo];
    const long long r = k - (long long)L * S.off[lo];
    const int l = (int)(r / ns);
    seg = lo * L + l;
    p = S.off[lo] + (r - (long long)l * ns);
}

__device__ __forceinline__ float weight_W(const GPre &G, const float *ampc, unsigned g, int L, int l,
                                          const double *T_sorted, long long p) {
    const double T = T_sorted ? T_sorted[p] : 1.0;
    return (float)(kTwoPi * (double)G.su * (double)G.sv * (double)ampc[(size_t)g * L + l] * (double)G.o * T);
}

__global__ void k_foot_keys(const GPre *__restrict__ gp, const float *__restrict__ ampc,
                            const unsigned *__restrict__ sorted, const double *__restrict__ T_sorted, Segs S,
                            long long n_rec, FootParams F, int drop_zero, unsigned long long *__restrict__ key,
                            unsigned *__restrict__ val) {
    const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n_rec) return;
    int seg;
    long long p;
    slot_decode(S, k, seg, p);
    const int l = seg % S.n_lambda;
    const unsigned g = sorted[p];
    const GPre &G = gp[g];
    float r1[3], r2[3], r3[3];
    cols_f32(G.q, r1, r2, r3);
    const Foot f = footprint(r1, r2, G.su, G.sv, F.rho, F.dzmax[l]);
    const float W = weight_W(G, ampc, g, S.n_lambda, l, T_sorted, p);
    unsigned rk = 0xFFFFFFFFu - __float_as_uint(f.R);  // decreasing radius
    if (drop_zero && W == 0.f) rk = 0xFFFFFFFFu;
    key[k] = ((unsigned long long)seg << 32) | rk;
    val[k] = (unsigned)p;
}

__global__ void k_gather(const unsigned long long *__restrict__ key, const unsigned *__restrict__ val,
                         const GPre *__restrict__ gp, const float *__restrict__ ampc,
                         const unsigned *__restrict__ sorted, const double *__restrict__ T_sorted, Segs S,
                         long long n_rec, FootParams F, int drop_zero, int backward, Rec *__restrict__ rec,
                         float *__restrict__ Rr, int *__restrict__ invrec, int *status) {
    const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n_rec) return;
    const int seg = (int)(key[k] >> 32);
    const long long n_all = S.off[S.n_scenes];
    if (!in_bounds(seg < S.n_scenes * S.n_lambda && (long long)val[k] < n_all, status)) return;
    const int l = seg % S.n_lambda;
    const long long p = val[k];
    const unsigned g = sorted[p];
    if (!in_bounds((long long)g < n_all, status)) return;
    const GPre &G = gp[g];
    float r1[3], r2[3], r3[3];
    cols_f32(G.q, r1, r2, r3);
    const Foot f = footprint(r1, r2, G.su, G.sv, F.rho, F.dzmax[l]);
    const float W = weight_W(G, ampc, g, S.n_lambda, l, T_sorted, p);
    const float ku = (float)(kKappa * (double)G.su), kv = (float)(kKappa * (double)G.sv);
    const float w3 = backward ? 1.f : W;
    Rec r;
    r.r1x = ku * r1[0];
    r.r1y = ku * r1[1];
    r.r1z = ku * r1[2];
    r.r2x = kv * r2[0];
    r.r2y = kv * r2[1];
    r.r2z = kv * r2[2];
    r.r3x = w3 * r3[0];
    r.r3y = w3 * r3[1];
    r.r3z = w3 * r3[2];
    r.mx = (float)(-kTwoPi * G.mu[0]);  // phase deltas in radians: -2 pi mu . (f - f0)
    r.my = (float)(-kTwoPi * G.mu[1]);
    r.mz = (float)(-kTwoPi * G.mu[2]);
    r.e00 = f.e00;
    r.e01 = f.e01;
    r.e11 = f.e11;
    r.W = W;
    r.mux = G.mu[0];
    r.muy = G.mu[1];
    r.muz = G.mu[2];
    r.g = (int)g;
    r.wz = f.wz;
    rec[k] = r;
    Rr[k] = (drop_zero && W == 0.f) ? -1.f : f.R;
    if (invrec) invrec[(size_t)g * S.n_lambda + l] = (int)k;
}

// inspection: footprint ellipse per input Gaussian for wavelength l
__global__ void k_foot_inspect(const GPre *__restrict__ gp, long long n, float rho, float dzmax,
                               float *__restrict__ out) {
    const long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= n) return;
    const GPre &G = gp[g];
    float r1[3], r2[3], r3[3];
    cols_f32(G.q, r1, r2, r3);
    const Foot f = footprint(r1, r2, G.su, G.sv, rho, dzmax);
    out[3 * g] = f.e00;
    out[3 * g + 1] = f.e01;
    out[3 * g + 2] = f.e11;
}

// algorithmic work: grid frequencies inside each (Gaussian, wavelength) footprint ellipse,
// counted row by row (the ellipse's chord on each row of the grid)
__global__ void k_count_pairs(const GPre *__restrict__ gp, long long n, int n_lambda, FootParams F, int H, int W,
                              double dfx, double dfy, unsigned long long *__restrict__ acc) {
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    unsigned long long cnt = 0;
    if (t < n * n_lambda) {
        const long long g = t / n_lambda;
        const int l = (int)(t % n_lambda);
        const GPre &G = gp[g];
        float r1[3], r2[3], r3[3];
        cols_f32(G.q, r1, r2, r3);
        const Foot f = footprint(r1, r2, G.su, G.sv, F.rho, F.dzmax[l]);
        const double e00 = f.e00, e01 = f.e01, e11 = f.e11;
        for (int r = 0; r < H; ++r) {
            const double fy = (double)(r - H / 2) * dfy;
            // e00 fx^2 + 2 e01 fy fx + e11 fy^2 <= 1
            long long c_lo, c_hi;
            if (e00 > 0) {
                const double disc = e01 * e01 * fy * fy - e00 * (e11 * fy * fy - 1.0);
                if (disc < 0) continue;
                const double sq = sqrt(disc);
                const double xa = (-e01 * fy - sq) / e00, xb = (-e01 * fy + sq) / e00;
                c_lo = (long long)ceil(xa / dfx) + W / 2;
                c_hi = (long long)floor(xb / dfx) + W / 2;
            } else {
                if (e11 * fy * fy > 1.0) continue;
                c_lo = 0;
                c_hi = W - 1;
            }
            c_lo = c_lo < 0 ? 0 : c_lo;
            c_hi = c_hi > W - 1 ? W - 1 : c_hi;
            if (c_hi >= c_lo) cnt += (unsigned long long)(c_hi - c_lo + 1);
        }
    }
    for (int o = 16; o > 0; o >>= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
    if ((threadIdx.x & 31) == 0 && cnt) atomicAdd(acc, cnt);
}

// work items: (segment, tile) -> number of leading records whose footprint radius reaches
// the tile (records are in decreasing-radius order); key orders items by decreasing work
// Items are ordered segment-major (one wavelength's records -- at most a few hundred MB --
// stay resident in L2 while all CTAs stream them), longest first inside a segment.
__global__ void k_items(const float *__restrict__ Rr, Segs S, int n_seg, int H, int W, int tw, int th, int tiles_x,
                        int n_tiles, double dfx, double dfy, unsigned long long *__restrict__ ikey,
                        unsigned *__restrict__ ival, int *__restrict__ icount) {
    const long long it = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (it >= (long long)n_seg * n_tiles) return;
    const int seg = (int)(it / n_tiles), tile = (int)(it % n_tiles);
    const int tx = tile % tiles_x, ty = tile / tiles_x;
    const int c_lo = tx * tw, c_hi = min(tx * tw + tw, W) - 1;
    const int r_lo = ty * th, r_hi = min(ty * th + th, H) - 1;
    const double x0 = (double)(c_lo - W / 2) * dfx, x1 = (double)(c_hi - W / 2) * dfx;
    const double y0 = (double)(r_lo - H / 2) * dfy, y1 = (double)(r_hi - H / 2) * dfy;
    const double nx = fmin(fmax(0.0, x0), x1), ny = fmin(fmax(0.0, y0), y1);
    const float rt = (float)(sqrt(nx * nx + ny * ny) * (1.0 - 1e-6));
    const long long base = seg_start(S, seg);
    long long lo = 0, hi = seg_size(S, seg);  // count of entries with R >= rt (R non-increasing)
    while (lo < hi) {
        const long long mid = (lo + hi) >> 1;
        if (Rr[base + mid] >= rt) lo = mid + 1;
        else hi = mid;
    }
    icount[it] = (int)lo;
    ikey[it] = ((unsigned long long)seg << 32) | (0xFFFFFFFFu - (unsigned)lo);
    ival[it] = (unsigned)it;
}

// ---------------------------------------------------------------------------------------
// centred inverse DFT around cuFFT:
//   u[r,c] = dfx dfy e^{j2pi(m0 r0/H + n0 c0/W)} e^{-j2pi(m0 r/H + n0 c/W)}
//            * IFFT_unnormalised( u_SLM[m,n] e^{-j2pi(m r0/H + n c0/W)} )[r,c],   m0 = r0 = H/2, n0 = c0 = W/2
// The pre-modulation is fused into the splats; this is the post-modulation, and the
// adjoint pair used by the backward.
// ---------------------------------------------------------------------------------------

template <typename R>
struct Cx;
template <>
struct Cx<float> {
    using T = float2;
};
template <>
struct Cx<double> {
    using T = double2;
};

// mode 0: forward post-modulation; 1: backward pre-modulation (conj of the post factor
// without the constant); 2: backward post-modulation (adjoint of the pre-modulation, with
// the constant and the scale)
template <typename R>
__device__ __forceinline__ void modulate_pixel(typename Cx<R>::T *__restrict__ data, int n_slices, int H, int W,
                                               double scale, int mode, int r, int c) {
    const long long hw = (long long)H * W;
    const int h2 = H / 2, w2 = W / 2;
    R sn, cs;
    R sc = (mode == 0 || mode == 2) ? (R)scale : (R)1;
    if (((H | W) & 1) == 0) {
        // even H, W: m0 r / H + n0 c / W = (r + c) / 2 cycles, so every factor is (-1)^(r + c), times
        // (-1)^(H/2 + W/2) for the origin term of modes 0 and 2 -- exact, no trigonometry
        const int k = r + c + ((mode == 0 || mode == 2) ? h2 + w2 : 0);
        sn = (R)0;
        cs = (k & 1) ? (R)-1 : (R)1;
    } else {
        // angle = num / (H W) cycles, num an exact integer (see mod_num2)
        long long num;
        if (mode == 0) {  // e^{j2pi(m0 r0/H + n0 c0/W)} e^{-j2pi(m0 r/H + n0 c/W)}
            num = mod_num2(h2, h2, 1, w2, w2, 1, H, W) - mod_num2(h2, r, 1, w2, c, 1, H, W);
        } else if (mode == 1) {  // e^{+j2pi(m0 r/H + n0 c/W)}
            num = mod_num2(h2, r, 1, w2, c, 1, H, W);
        } else if (mode == 2) {  // e^{-j2pi(m0 r0/H + n0 c0/W)} e^{+j2pi(m r0/H + n c0/W)}
            num = mod_num2(r, h2, 1, c, w2, 1, H, W) - mod_num2(h2, h2, 1, w2, w2, 1, H, W);
        } else {  // forward pre-modulation e^{-j2pi(m r0/H + n c0/W)} (natural-layout spectrum -> cuFFT input)
            num = -mod_num2(r, h2, 1, c, w2, 1, H, W);
        }
        if (num < 0) num += hw;
        if (2 * num > hw) num -= hw;  // |angle| <= 1/2 cycle
        if (sizeof(R) == 8) {
            double s8, c8;
            sincospi(2.0 * (double)num / (double)hw, &s8, &c8);
            sn = (R)s8;
            cs = (R)c8;
        } else {
            float s4, c4;
            sincospif(2.0f * (float)num * (1.0f / (float)hw), &s4, &c4);
            sn = (R)s4;
            cs = (R)c4;
        }
    }
    sn *= sc;
    cs *= sc;
    typename Cx<R>::T *p = data + (size_t)r * W + c;
#pragma unroll 4
    for (int sl = 0; sl < n_slices; ++sl) {
        typename Cx<R>::T v = p[(size_t)sl * hw];
        const R re = v.x * cs - v.y * sn;
        v.y = v.x * sn + v.y * cs;
        v.x = re;
        p[(size_t)sl * hw] = v;
    }
}

template <typename R>
__global__ void k_modulate(typename Cx<R>::T *__restrict__ data, int n_slices, int H, int W, double scale, int mode) {
    // one thread per (row, column): the factor is the same in every slice; rows stride by gridDim.y
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= W) return;
    for (int r = blockIdx.y; r < H; r += gridDim.y) modulate_pixel<R>(data, n_slices, H, W, scale, mode, r, c);
}


// ---------------------------------------------------------------------------------------
// double-phase encoding (supplement, phase encoding; the garbled formula read as
// P1,2 = phi -/+ acos(a))
// ---------------------------------------------------------------------------------------

template <typename R>
__global__ void k_amax(const typename Cx<R>::T *__restrict__ f, long long hw, unsigned long long *__restrict__ amax2) {
    const int l = blockIdx.y;
    const typename Cx<R>::T *fl = f + (size_t)l * hw;
    const long long stride = (long long)gridDim.x * blockDim.x;
    R m0 = 0, m1 = 0, m2 = 0, m3 = 0;  // four loads in flight per thread
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    for (; i + 3 * stride < hw; i += 4 * stride) {
        const typename Cx<R>::T v0 = fl[i], v1 = fl[i + stride], v2 = fl[i + 2 * stride], v3 = fl[i + 3 * stride];
        m0 = fmax(m0, v0.x * v0.x + v0.y * v0.y);
        m1 = fmax(m1, v1.x * v1.x + v1.y * v1.y);
        m2 = fmax(m2, v2.x * v2.x + v2.y * v2.y);
        m3 = fmax(m3, v3.x * v3.x + v3.y * v3.y);
    }
    for (; i < hw; i += stride) {
        const typename Cx<R>::T v = fl[i];
        m0 = fmax(m0, v.x * v.x + v.y * v.y);
    }
    R m = fmax(fmax(m0, m1), fmax(m2, m3));
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) {
        unsigned long long bits =
            sizeof(R) == 8 ? (unsigned long long)__double_as_longlong((double)m) : (unsigned long long)__float_as_uint((float)m);
        atomicMax(&amax2[l], bits);
    }
}

// DPAC (Sec. 5): one wavelength per grid row y, 32-bit pixel indices (H W < 2^31 is checked by
// the API), four pixels per thread.
template <typename R>
__global__ void k_dpac(const typename Cx<R>::T *__restrict__ f, int H, int W,
                       const unsigned long long *__restrict__ amax2, double amp_scale, float *__restrict__ out) {
    const int l = blockIdx.y;
    const unsigned hw = (unsigned)H * (unsigned)W;
    const R pi = (R)kPi, tpi = (R)kTwoPi, inv_tpi = (R)(1.0 / kTwoPi);
    R m2max;
    if (amp_scale > 0) m2max = (R)(amp_scale * amp_scale);
    else if (sizeof(R) == 8) m2max = (R)__longlong_as_double((long long)amax2[l]);
    else m2max = (R)__uint_as_float((unsigned)amax2[l]);
    const R inv_m2 = m2max > 0 ? (R)1 / m2max : (R)0;
    const typename Cx<R>::T *fl = f + (size_t)l * hw;
    float *ol = out + (size_t)l * hw;
#pragma unroll
    for (int u = 0; u < 4; ++u) {
        const unsigned pix = ((unsigned)blockIdx.x * 4u + (unsigned)u) * blockDim.x + threadIdx.x;
        if (pix >= hw) break;
        const unsigned r = pix / (unsigned)W, c = pix - r * (unsigned)W;
        const typename Cx<R>::T v = fl[pix];
        const R m2 = v.x * v.x + v.y * v.y;
        R a = sqrt(m2 * inv_m2);
        a = a > (R)1 ? (R)1 : a;
        const R phi = atan2(v.y, v.x);
        const R ac = acos(a);
        R p = ((r + c) & 1u) == 0 ? phi - ac : phi + ac;
        p = p - tpi * floor((p + pi) * inv_tpi);
        if (p < -pi) p += tpi;
        if (p >= pi) p -= tpi;
        ol[pix] = (float)p;
    }
}

// ---------------------------------------------------------------------------------------
// host launchers
// ---------------------------------------------------------------------------------------

static inline unsigned nblk(long long n, int t) { return (unsigned)((n + t - 1) / t); }

cudaError_t launch_prep(const SceneTable &T, long long n_total, GPre *gp, float *ampc, unsigned long long *dkey,
                        unsigned *dval, int *status, cudaStream_t s) {
    if (n_total <= 0) return cudaSuccess;
    k_prep<<<nblk(n_total, 256), 256, 0, s>>>(T, n_total, gp, ampc, dkey, dval, status);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_scene_key(const GPre *gp, const unsigned *sorted, long long n, unsigned *skey, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    k_scene_key<<<nblk(n, 256), 256, 0, s>>>(gp, sorted, n, skey);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_transmittance(const GPre *gp, const unsigned *sorted, const Segs &S, long long n, double alpha_min,
                                 TData *td, double *T_sorted, double *T_g, TQuery *tq, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    k_tdata<<<nblk(n, 256), 256, 0, s>>>(gp, sorted, n, alpha_min, td);
    k_transmit<<<nblk(n, kTChunk), kTChunk, 0, s>>>(td, sorted, S, n, alpha_min, T_sorted, T_g, tq);
    count_launches(2);
    return cudaGetLastError();
}

cudaError_t launch_tgrad(const TData *td, TQuery *tq, const GPre *gp, const unsigned *sorted, const double *dT_g,
                         const float *quat_in, const Segs &S, long long n, double alpha_min, double *dmean,
                         float *dquat, float *dscale, float *dopacity, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    k_tq_dT<<<nblk(n, 256), 256, 0, s>>>(sorted, dT_g, n, tq);
    k_tgrad_query<<<nblk(n, kTChunk), kTChunk, 0, s>>>(td, tq, sorted, S, n, alpha_min, dmean);
    k_tgrad_front<<<nblk(n, kTChunk), kTChunk, 0, s>>>(td, tq, gp, sorted, quat_in, S, n, alpha_min, dmean, dquat,
                                                         dscale, dopacity);
    count_launches(3);
    return cudaGetLastError();
}

cudaError_t launch_rec64(const GPre *gp, const float *ampc, const unsigned *sorted, const double *T_sorted, long long n,
                         int L, Rec64 *rec, double *w, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    k_rec64<<<nblk(n, 256), 256, 0, s>>>(gp, ampc, sorted, T_sorted, n, L, rec, w);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_foot_keys(const GPre *gp, const float *ampc, const unsigned *sorted, const double *T_sorted,
                             const Segs &S, long long n_rec, const FootParams &F, int drop_zero,
                             unsigned long long *key, unsigned *val, cudaStream_t s) {
    if (n_rec <= 0) return cudaSuccess;
    k_foot_keys<<<nblk(n_rec, 256), 256, 0, s>>>(gp, ampc, sorted, T_sorted, S, n_rec, F, drop_zero, key, val);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_gather(const unsigned long long *key, const unsigned *val, const GPre *gp, const float *ampc,
                          const unsigned *sorted, const double *T_sorted, const Segs &S, long long n_rec,
                          const FootParams &F, int drop_zero, int backward, Rec *rec, float *Rr, int *invrec,
                          int *status, cudaStream_t s) {
    if (n_rec <= 0) return cudaSuccess;
    k_gather<<<nblk(n_rec, 256), 256, 0, s>>>(key, val, gp, ampc, sorted, T_sorted, S, n_rec, F, drop_zero, backward,
                                               rec, Rr, invrec, status);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_foot_inspect(const GPre *gp, long long n, float rho, float dzmax, float *out, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    k_foot_inspect<<<nblk(n, 256), 256, 0, s>>>(gp, n, rho, dzmax, out);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_items(const float *Rr, const Segs &S, int n_seg, int H, int W, int tw, int th, int tiles_x,
                         int n_tiles, double dfx, double dfy, unsigned long long *ikey, unsigned *ival, int *icount,
                         cudaStream_t s) {
    const long long n = (long long)n_seg * n_tiles;
    k_items<<<nblk(n, 256), 256, 0, s>>>(Rr, S, n_seg, H, W, tw, th, tiles_x, n_tiles, dfx, dfy, ikey, ival, icount);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_count_pairs(const GPre *gp, long long n, int n_lambda, const FootParams &F, int H, int W,
                               double dfx, double dfy, unsigned long long *acc, cudaStream_t s) {
    const long long t = n * n_lambda;
    if (t <= 0) return cudaSuccess;
    k_count_pairs<<<nblk(t, 256), 256, 0, s>>>(gp, n, n_lambda, F, H, W, dfx, dfy, acc);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_modulate(void *data, int prec64, int n_slices, int H, int W, double scale, int mode,
                            cudaStream_t s) {
    const long long n = (long long)n_slices * H * W;
    if (n <= 0) return cudaSuccess;
    const dim3 grid(nblk(W, 256), (unsigned)std::min(H, 65535));
    if (prec64)
        k_modulate<double><<<grid, 256, 0, s>>>((double2 *)data, n_slices, H, W, scale, mode);
    else
        k_modulate<float><<<grid, 256, 0, s>>>((float2 *)data, n_slices, H, W, scale, mode);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_encode(const void *field, int prec64, int n_lambda, int H, int W, unsigned long long *amax2,
                          double amp_scale, float *out, cudaStream_t s) {
    const long long hw = (long long)H * W;
    if (amp_scale <= 0) {
        cudaError_t e = cudaMemsetAsync(amax2, 0, sizeof(unsigned long long) * n_lambda, s);
        if (e != cudaSuccess) return e;
        const unsigned gx = (unsigned)std::min<long long>(nblk(hw, 256), 608);
        if (prec64)
            k_amax<double><<<dim3(gx, n_lambda), 256, 0, s>>>((const double2 *)field, hw, amax2);
        else
            k_amax<float><<<dim3(gx, n_lambda), 256, 0, s>>>((const float2 *)field, hw, amax2);
        count_launches(1);
    }
    const dim3 grid(nblk(hw, 1024), (unsigned)n_lambda);
    if (prec64)
        k_dpac<double><<<grid, 256, 0, s>>>((const double2 *)field, H, W, amax2, amp_scale, out);
    else
        k_dpac<float><<<grid, 256, 0, s>>>((const float2 *)field, H, W, amax2, amp_scale, out);
    count_launches(1);
    return cudaGetLastError();
}

}  // namespace gws
