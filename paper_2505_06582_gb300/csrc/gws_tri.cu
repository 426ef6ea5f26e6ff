// gws_tri.cu -- the triangle primitive of the supplement's section on polygon-based methods:
// Eq. 10 with the canonical Gaussian replaced by the canonical triangle P = {(0,0), (1,0), (1,1)},
// the 2D affine map A = [[1,1],[0,1]] V_o^-1 (affine theorem of Eq. 8: factor |det V_o|, argument
// A^-T k_o) and the translation mu = v1, summed over triangles as in Eq. 12:
//   u_hat(f) = c o |r3 . f| / f_z |det V_o| T(A^-T (r1 . d, r2 . d)) e^{-j 2 pi f . v1},  d = f - f_r.
// T(nu) = int_P e^{-j 2 pi nu . x} dx is the second divided difference of exp at the vertex
// phases z = j (0, -a, -(a + b)), a = 2 pi nu_x, b = 2 pi nu_y, evaluated in FP32 as
//   (E[t1,t2] - E[t0,t1]) / (j (t2 - t0)),  E[p,q] = e^{j (p+q)/2} sin((q-p)/2) / ((q-p)/2)
// (the record's phase added to (p+q)/2 before the cis; one approximate reciprocal for both sincs
// and the 1 / (t2 - t0): 7 MUFU operations per pair),
// with t0 <= t1 <= t2 the sorted phases when their spread exceeds TRI_SPREAD, else as the series
// e^{j tbar} sum_k j^k h_k(t - tbar) / (k+2)! (h_k the complete homogeneous polynomials).
// Dense: the spectrum of a triangle has no compact footprint.  One CTA per (tile, wavelength);
// triangles stream through shared memory in chunks with per-(triangle, tile) FP64 phase anchors.
#include "gws_prep.h"

namespace gws {

constexpr int TTW = 32, TTH = 16, TNT = 256;  // 2 pixels (columns c, c + 16) per thread, one f32x2 pair
constexpr float TRI_SPREAD = 0.5f;

__global__ void k_tri_prep(const double *__restrict__ v, const float *__restrict__ opacity,
                           const float *__restrict__ amp, long long n, int L, TriRec *__restrict__ rec,
                           float *__restrict__ w, int *__restrict__ status) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double *p = v + 9 * i;
    double e2[3], e3[3];
    for (int k = 0; k < 3; ++k) {
        e2[k] = p[3 + k] - p[k];
        e3[k] = p[6 + k] - p[k];
    }
    bool fin = true;
    for (int k = 0; k < 9; ++k) fin = fin && isfinite(p[k]);
    const double n2 = sqrt(e2[0] * e2[0] + e2[1] * e2[1] + e2[2] * e2[2]);
    double nr[3] = {e2[1] * e3[2] - e2[2] * e3[1], e2[2] * e3[0] - e2[0] * e3[2], e2[0] * e3[1] - e2[1] * e3[0]};
    const double nn = sqrt(nr[0] * nr[0] + nr[1] * nr[1] + nr[2] * nr[2]);
    const double n3 = sqrt(e3[0] * e3[0] + e3[1] * e3[1] + e3[2] * e3[2]);
    const float o = opacity[i];
    TriRec r;
    // degenerate: an edge of zero length or the edges (nearly) parallel (sine of their angle < 1e-9)
    if (!fin || !(n2 > 0.0) || !(nn > 1e-9 * n2 * n3) || !isfinite(o)) {
        atomicOr(status, fin && isfinite(o) ? ST_BADVALUE : ST_NONFINITE);
        for (int k = 0; k < 6; ++k) r.M[k] = 0.f;
        r.r3[0] = r.r3[1] = r.r3[2] = 0.f;
        r.v1[0] = r.v1[1] = r.v1[2] = 0.0;
        rec[i] = r;
        for (int l = 0; l < L; ++l) w[i * L + l] = 0.f;
        return;
    }
    double r1[3], r3[3], r2[3];
    for (int k = 0; k < 3; ++k) {
        r1[k] = e2[k] / n2;
        r3[k] = nr[k] / nn;
    }
    r2[0] = r3[1] * r1[2] - r3[2] * r1[1];
    r2[1] = r3[2] * r1[0] - r3[0] * r1[2];
    r2[2] = r3[0] * r1[1] - r3[1] * r1[0];
    // V_o = [[p, q], [0, s]] (columns: vertices 2 and 3 in the triangle's frame), A = [[1,1],[0,1]] V_o^-1
    const double vp = n2, vq = r1[0] * e3[0] + r1[1] * e3[1] + r1[2] * e3[2];
    const double vs = r2[0] * e3[0] + r2[1] * e3[1] + r2[2] * e3[2];
    // A^-1 = V_o [[1,1],[0,1]]^-1 = [[p, q - p], [0, s]], so A^-T = [[p, 0], [q - p, s]]
    const double ait[2][2] = {{vp, 0.0}, {vq - vp, vs}};
    for (int k = 0; k < 3; ++k) {
        r.M[k] = (float)(ait[0][0] * r1[k] + ait[0][1] * r2[k]);
        r.M[3 + k] = (float)(ait[1][0] * r1[k] + ait[1][1] * r2[k]);
        r.r3[k] = (float)r3[k];
        r.v1[k] = p[k];
    }
    rec[i] = r;
    const double det = vp * vs;  // |det V_o| (s > 0 by construction)
    for (int l = 0; l < L; ++l) w[i * L + l] = (float)(det * (double)o * (double)amp[i * L + l]);
}

// e^{j x} for |x| up to a few thousand radians: x - 2 pi round(x / 2 pi) first (FP32 rounding trick)
__device__ __forceinline__ float2 cis_reduced(float x) {
    const float k = __fadd_rn(fmaf(x, 0.15915494309189535f, 12582912.0f), -12582912.0f);
    const float r = fmaf(k, -6.28318530717958647692f, x);
    return make_float2(cos_approx(r), sin_approx(r));
}

// sin(h) / h for h >= 0 as a fraction (num, den): (sin h, h) with the argument reduced to
// [-pi, pi] first, or (1, 1) below 1e-4 (where 1 - h^2 / 6 rounds to 1)
__device__ __forceinline__ float2 sinc_frac(float h) {
    if (!(h > 1e-4f)) return make_float2(1.f, 1.f);
    const float k = __fadd_rn(fmaf(h, 0.15915494309189535f, 12582912.0f), -12582912.0f);
    return make_float2(sin_approx(fmaf(k, -6.28318530717958647692f, h)), h);
}

// T(nu) e^{j th} of the canonical triangle from its sorted vertex phases t0 <= t1 <= t2 (z = j t)
// and the record's phase th (both factors' phases are added before the one cis per term)
__device__ __forceinline__ float2 tri_canonical_phased(float t0, float t1, float t2, float th) {
    const float sp = t2 - t0;
    if (sp > TRI_SPREAD) {
        // E[p,q] e^{j th} = e^{j ((p+q)/2 + th)} sinc((q-p)/2); the two sincs and 1 / sp share one
        // reciprocal: (n12 d01 c12 - n01 d12 c01) / (d12 d01 sp)
        const float2 f12 = sinc_frac(0.5f * (t2 - t1)), f01 = sinc_frac(0.5f * (t1 - t0));
        const float2 c12 = cis_reduced(fmaf(0.5f, t1 + t2, th)), c01 = cis_reduced(fmaf(0.5f, t0 + t1, th));
        const float w12 = f12.x * f01.y, w01 = f01.x * f12.y;
        const float dr = fmaf(w12, c12.x, -w01 * c01.x), di = fmaf(w12, c12.y, -w01 * c01.y);
        const float inv = __fdividef(1.f, f12.y * f01.y * sp);  // (dr + j di) / (j sp) = (di - j dr) / sp
        return make_float2(di * inv, -dr * inv);
    }
    const float tb = (t0 + t1 + t2) * (1.f / 3.f);
    const float u0 = t0 - tb, u1 = t1 - tb, u2 = t2 - tb;
    // h_k(u0) = u0^k, h_k(u0,u1) = h_k(u0) + u1 h_{k-1}(u0,u1), h_k(u0,u1,u2) = h_k(u0,u1) + u2 h_{k-1}(...)
    float a = 1.f, b = 1.f, c = 1.f;
    float re = 0.5f, im = 0.f;  // k = 0: 1 / 2!
    float inv_fact = 0.5f;
#pragma unroll
    for (int k = 1; k < 8; ++k) {
        a *= u0;
        b = fmaf(u1, b, a);
        c = fmaf(u2, c, b);
        inv_fact *= 1.f / (float)(k + 2);  // 1 / (k + 2)!, folded at compile time
        const float t = c * inv_fact;
        switch (k & 3) {  // j^k
            case 0: re += t; break;
            case 1: im += t; break;
            case 2: re -= t; break;
            default: im -= t; break;
        }
    }
    const float2 e = cis_reduced(tb + th);
    return make_float2(re * e.x - im * e.y, re * e.y + im * e.x);
}

// The thread's two pixels as one f32x2 pair (h = 0, 1): sin(h)/h as (num, den) per pixel
__device__ __forceinline__ void sinc_frac2(float2 h, float2 &num, float2 &den) {
    const float2 k = __fadd2_rn(__ffma2_rn(h, pair(0.15915494309189535f), pair(12582912.0f)), pair(-12582912.0f));
    const float2 a = __ffma2_rn(k, pair(-6.28318530717958647692f), h);
    const bool bx = h.x > 1e-4f, by = h.y > 1e-4f;
    num = make_float2(bx ? sin_approx(a.x) : 1.f, by ? sin_approx(a.y) : 1.f);
    den = make_float2(bx ? h.x : 1.f, by ? h.y : 1.f);
}

// e^{j x} of both pixels: x - 2 pi round(x / 2 pi) first
__device__ __forceinline__ void cis2(float2 x, float2 &re, float2 &im) {
    const float2 k = __fadd2_rn(__ffma2_rn(x, pair(0.15915494309189535f), pair(12582912.0f)), pair(-12582912.0f));
    const float2 r = __ffma2_rn(k, pair(-6.28318530717958647692f), x);
    re = make_float2(cos_approx(r.x), cos_approx(r.y));
    im = make_float2(sin_approx(r.x), sin_approx(r.y));
}

struct TriConst {  // per (triangle, tile), FP32 except the anchor
    float nu0x, nu0y, mxx, mxy, mxz, myx, myy, myz;  // nu = nu0 + M (dx, dy, dz)
    float g0, r3x, r3y, r3z;                         // r3 . f = g0 + r3 . delta
    float th0, tx, ty, tz;                           // phase = th0 + (tx dx + ty dy + tz dz)
    float w;
};

__global__ void __launch_bounds__(TNT, 4) k_splat_tri(const TriRec *__restrict__ rec, const float *__restrict__ wgt,
                                                      long long n, int L, int H, int W, double dfx, double dfy,
                                                      InvLam il, int field_mode, int phase_match,
                                                      float2 *__restrict__ out) {
    __shared__ TriConst S[TNT];
    const int tiles_x = (W + TTW - 1) / TTW;
    const int tx = blockIdx.x % tiles_x, ty = blockIdx.x / tiles_x, l = blockIdx.y;
    const int c_lo = tx * TTW, r_lo = ty * TTH;
    const int c_hi = min(c_lo + TTW, W) - 1, r_hi = min(r_lo + TTH, H) - 1;
    const double inv_lam = il.v[l], k2 = inv_lam * inv_lam;
    int c_ref, r_ref;
    tile_ref(c_lo, c_hi, r_lo, r_hi, H, W, dfx, dfy, k2, c_ref, r_ref);
    const double f0x = (double)(c_ref - W / 2) * dfx, f0y = (double)(r_ref - H / 2) * dfy;
    const double f0z = sqrt(fmax(k2 - (f0x * f0x + f0y * f0y), 0.0));
    const int tid = threadIdx.x;
    const int row = r_lo + tid / 16;
    float dx[2], dz[2], ifz[2];
    float2 acc_re = make_float2(0.f, 0.f), acc_im = make_float2(0.f, 0.f);
    float sum_re[2] = {0.f, 0.f}, sum_im[2] = {0.f, 0.f}, cmp_re[2] = {0.f, 0.f}, cmp_im[2] = {0.f, 0.f};
    bool ok[2];
    const double fy = (double)(row - H / 2) * dfy;
    const float dy = (float)((double)(row - r_ref) * dfy);
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const int col = c_lo + (tid % 16) + 16 * h;
        const double fx = (double)(col - W / 2) * dfx;
        const double rho2 = fx * fx + fy * fy;
        ok[h] = row < H && col < W && rho2 < k2;
        const double fz = ok[h] ? sqrt(k2 - rho2) : 1.0;
        dx[h] = (float)((double)(col - c_ref) * dfx);
        dz[h] = ok[h] ? (float)(fz - f0z) : 0.f;
        ifz[h] = ok[h] ? (float)(1.0 / fz) : 0.f;
    }
    for (long long c0 = 0; c0 < n; c0 += TNT) {
        const int nc = (int)min((long long)TNT, n - c0);
        __syncthreads();
        if (tid < nc) {
            const TriRec r = rec[c0 + tid];
            TriConst &T = S[tid];
            const double d0z = f0z - inv_lam;  // d = f - f_r at the tile reference
            T.nu0x = (float)(r.M[0] * f0x + r.M[1] * f0y + r.M[2] * d0z);
            T.nu0y = (float)(r.M[3] * f0x + r.M[4] * f0y + r.M[5] * d0z);
            T.mxx = r.M[0];
            T.mxy = r.M[1];
            T.mxz = r.M[2];
            T.myx = r.M[3];
            T.myy = r.M[4];
            T.myz = r.M[5];
            T.g0 = (float)(r.r3[0] * f0x + r.r3[1] * f0y + r.r3[2] * f0z);
            T.r3x = r.r3[0];
            T.r3y = r.r3[1];
            T.r3z = r.r3[2];
            double cyc = -(f0x * r.v1[0] + f0y * r.v1[1] + f0z * r.v1[2]);
            if (phase_match) cyc += r.v1[2] * inv_lam;
            cyc -= rint(cyc);
            T.th0 = (float)(kTwoPi * cyc);
            T.tx = (float)(-kTwoPi * r.v1[0]);
            T.ty = (float)(-kTwoPi * r.v1[1]);
            T.tz = (float)(-kTwoPi * r.v1[2]);
            T.w = wgt[(c0 + tid) * L + l];
        }
        __syncthreads();
        const float2 dxp = make_float2(dx[0], dx[1]), dzp = make_float2(dz[0], dz[1]);
        const float2 ifzp = make_float2(ifz[0], ifz[1]);
        for (int k = 0; k < nc; ++k) {
            const TriConst &T = S[k];
            // the row's share of the four affine forms, once per (triangle, thread); then both
            // pixels as one packed f32x2 pair
            const float2 bx = pair(fmaf(T.mxy, dy, T.nu0x)), by = pair(fmaf(T.myy, dy, T.nu0y));
            const float2 bg = pair(fmaf(T.r3y, dy, T.g0)), bt = pair(fmaf(T.ty, dy, T.th0));
            const float2 nx = __ffma2_rn(pair(T.mxz), dzp, __ffma2_rn(pair(T.mxx), dxp, bx));
            const float2 ny = __ffma2_rn(pair(T.myz), dzp, __ffma2_rn(pair(T.myx), dxp, by));
            const float2 th = __ffma2_rn(pair(T.tz), dzp, __ffma2_rn(pair(T.tx), dxp, bt));
            const float2 ga = __ffma2_rn(pair(T.r3z), dzp, __ffma2_rn(pair(T.r3x), dxp, bg));
            // vertex phases of e^{-j 2 pi nu . x} at (0,0), (1,0), (1,1): 0, -a, -(a + b), sorted
            const float2 p1 = __fmul2_rn(nx, pair(-6.28318530717958647692f));
            const float2 p2 = __fmul2_rn(__fadd2_rn(nx, ny), pair(-6.28318530717958647692f));
            const float2 t0 = make_float2(fminf(0.f, fminf(p1.x, p2.x)), fminf(0.f, fminf(p1.y, p2.y)));
            const float2 t2 = make_float2(fmaxf(0.f, fmaxf(p1.x, p2.x)), fmaxf(0.f, fmaxf(p1.y, p2.y)));
            const float2 t1 = __fadd2_rn(__fadd2_rn(p1, p2), make_float2(-(t0.x + t2.x), -(t0.y + t2.y)));
            const float2 sp = __fadd2_rn(t2, make_float2(-t0.x, -t0.y));
            float2 vre, vim;
            if (sp.x > TRI_SPREAD && sp.y > TRI_SPREAD) {
                // E[p,q] e^{j th} = e^{j ((p+q)/2 + th)} sinc((q-p)/2), one reciprocal per pixel
                float2 n12, d12, n01, d01, c12r, c12i, c01r, c01i;
                sinc_frac2(__fmul2_rn(__fadd2_rn(t2, make_float2(-t1.x, -t1.y)), pair(0.5f)), n12, d12);
                sinc_frac2(__fmul2_rn(__fadd2_rn(t1, make_float2(-t0.x, -t0.y)), pair(0.5f)), n01, d01);
                cis2(__ffma2_rn(pair(0.5f), __fadd2_rn(t1, t2), th), c12r, c12i);
                cis2(__ffma2_rn(pair(0.5f), __fadd2_rn(t0, t1), th), c01r, c01i);
                const float2 w12 = __fmul2_rn(n12, d01), w01 = __fmul2_rn(n01, d12);
                const float2 q1 = __fmul2_rn(w01, c01r), q2 = __fmul2_rn(w01, c01i);
                const float2 dr = __ffma2_rn(w12, c12r, make_float2(-q1.x, -q1.y));
                const float2 di = __ffma2_rn(w12, c12i, make_float2(-q2.x, -q2.y));
                const float2 den = __fmul2_rn(__fmul2_rn(d12, d01), sp);
                const float2 inv = make_float2(__fdividef(1.f, den.x), __fdividef(1.f, den.y));
                vre = __fmul2_rn(di, inv);  // (dr + j di) / (j sp) = (di - j dr) / sp
                vim = __fmul2_rn(make_float2(-dr.x, -dr.y), inv);
            } else {  // a pixel near the spectrum's centre: each pixel on its own branch
                const float2 v0 = tri_canonical_phased(t0.x, t1.x, t2.x, th.x);
                const float2 v1 = tri_canonical_phased(t0.y, t1.y, t2.y, th.y);
                vre = make_float2(v0.x, v1.x);
                vim = make_float2(v0.y, v1.y);
            }
            const float2 sw = __fmul2_rn(pair(T.w), __fmul2_rn(make_float2(fabsf(ga.x), fabsf(ga.y)), ifzp));
            acc_re = __ffma2_rn(sw, vre, acc_re);
            acc_im = __ffma2_rn(sw, vim, acc_im);
        }
        const float are[2] = {acc_re.x, acc_re.y}, aim[2] = {acc_im.x, acc_im.y};
#pragma unroll
        for (int h = 0; h < 2; ++h) {  // TwoSum-compensated merge of the chunk
            float t = sum_re[h] + are[h], bp = t - sum_re[h];
            cmp_re[h] += (sum_re[h] - (t - bp)) + (are[h] - bp);
            sum_re[h] = t;
            t = sum_im[h] + aim[h];
            bp = t - sum_im[h];
            cmp_im[h] += (sum_im[h] - (t - bp)) + (aim[h] - bp);
            sum_im[h] = t;
        }
        acc_re = acc_im = make_float2(0.f, 0.f);
    }
    if (row >= H) return;
    const long long hw = (long long)H * W;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const int col = c_lo + (tid % 16) + 16 * h;
        if (col >= W) continue;
        float re = ok[h] ? sum_re[h] + cmp_re[h] : 0.f, im = ok[h] ? sum_im[h] + cmp_im[h] : 0.f;
        if (field_mode) {  // centred-DFT pre-modulation e^{-j 2 pi (m r0 / H + n c0 / W)}
            if (((H | W) & 1) == 0) {  // even grid: (-1)^(r + c) exactly
                if ((row + col) & 1) {
                    re = -re;
                    im = -im;
                }
            } else {
                long long num = mod_num2(row, H / 2, 1, col, W / 2, 1, H, W);
                if (2 * num > hw) num -= hw;
                float sn, cs;
                sincospif(-2.0f * (float)num / (float)hw, &sn, &cs);
                const float r2 = re * cs - im * sn;
                im = re * sn + im * cs;
                re = r2;
            }
        }
        out[(size_t)l * hw + (size_t)row * W + col] = make_float2(re, im);
    }
}

cudaError_t launch_tri_prep(const double *v, const float *opacity, const float *amp, long long n, int L, TriRec *rec,
                            float *w, int *status, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    k_tri_prep<<<(unsigned)((n + 127) / 128), 128, 0, s>>>(v, opacity, amp, n, L, rec, w, status);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_splat_tri(const TriRec *rec, const float *w, long long n, int L, int H, int W, double dfx,
                             double dfy, const InvLam &il, int field_mode, int phase_match, float2 *out,
                             cudaStream_t s) {
    const int tiles = ((W + TTW - 1) / TTW) * ((H + TTH - 1) / TTH);
    k_splat_tri<<<dim3(tiles, L), TNT, 0, s>>>(rec, w, n, L, H, W, dfx, dfy, il, field_mode, phase_match, out);
    count_launches(1);
    return cudaGetLastError();
}

}  // namespace gws
