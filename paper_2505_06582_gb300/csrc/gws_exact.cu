// gws_exact.cu -- exact alpha wave blending (Eq. 5-6 with the spatial transmittance map,
// Algorithm S2), front to back over depth-ordered batches of Gaussians, and the batches of
// partially coherent GWS (Eq. 14; see the kernels after k_exact_accum):
//   u_k = the Gaussian's field on its own depth plane (Eq. 10 with the depth of the mean
//         set to zero, then the inverse DFT; produced by the batched forward),
//   u_SLM(f) += c_k o_k F(T u_k)(f) H(f, -z_k),   H(f, z) = exp(j 2 pi z f_z),
//   alpha_k = o_k |u_k| kept where > t_eps (or 1 where > t_binarize, else 0), T *= 1 - alpha_k.
// The batch's fields are masked in depth order per pixel (k_exact_mask), taken back to the
// spectrum by a centred forward DFT (cuFFT + modulations, scale px py), and accumulated with
// their propagators by k_exact_accum (per-(tile, Gaussian) FP64 phase anchors, FP32 deltas).
#include "gws_prep.h"

namespace gws {

__global__ void k_exact_gather(const unsigned *__restrict__ sorted, long long b0, int nb, const double *__restrict__ mean,
                               const float *__restrict__ quat, const float *__restrict__ scale,
                               const float *__restrict__ opacity, const float *__restrict__ amp, int L, ExactBatch E,
                               int pc) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= nb) return;
    const long long i = sorted[b0 + k];
    if (!in_bounds(b0 + k < E.n && i < E.n, E.status)) return;  // checking build only
    // the field on the Gaussian's own plane; partial coherence: at the origin (translated after the kernel)
    E.mean[3 * k] = pc ? 0.0 : mean[3 * i];
    E.mean[3 * k + 1] = pc ? 0.0 : mean[3 * i + 1];
    E.mean[3 * k + 2] = 0.0;
    if (pc)
        for (int c = 0; c < 3; ++c) E.mu[3 * k + c] = mean[3 * i + c];
    {  // the one-Gaussian record of k_single_spectra (c = o = T = 1)
        double q[4] = {quat[4 * i], quat[4 * i + 1], quat[4 * i + 2], quat[4 * i + 3]};
        const double qn = sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
        for (int m = 0; m < 4; ++m) q[m] /= qn;
        double r1[3], r2[3], r3[3];
        quat_cols<double>(q, r1, r2, r3);
        const double su = scale[2 * i], sv = scale[2 * i + 1];
        const double ku = kKappa * su, kv = kKappa * sv, w = kTwoPi * su * sv;
        for (int m = 0; m < 3; ++m) {
            E.rr[9 * k + m] = (float)(ku * r1[m]);
            E.rr[9 * k + 3 + m] = (float)(kv * r2[m]);
            E.rr[9 * k + 6 + m] = (float)(w * r3[m]);
        }
    }
    for (int m = 0; m < 4; ++m) E.quat[4 * k + m] = quat[4 * i + m];
    E.scale[2 * k] = scale[2 * i];
    E.scale[2 * k + 1] = scale[2 * i + 1];
    E.opacity[k] = 1.f;
    for (int l = 0; l < L; ++l) {
        E.amp[k * L + l] = 1.f;
        E.co[k * L + l] = amp[i * L + l] * opacity[i];
    }
    E.zk[k] = mean[3 * i + 2];
    E.ok[k] = opacity[i];
}

// The batch's fields at their own planes, in spectrum form: Eq. 10 for each one-Gaussian scene
// (c = o = T = 1, the mean from the gather) at every grid frequency -- no footprint truncation --
// times the centred-DFT pre-modulation, ready for one batched inverse FFT.  One CTA per (64 x 32
// tile, batch slot k, wavelength l): FP64 record and phase anchor at the tile's reference
// frequency, FP32 deltas per pixel (the per-pixel table gives f_z - f0_z and log2(1/f_z)).
constexpr int SKB = 8;  // one-Gaussian scenes per CTA of k_single_spectra

__global__ void __launch_bounds__(256) k_single_spectra(ExactBatch E, int nb, int L, int H, int W, double dfx,
                                                        double dfy, InvLam il, const float2 *__restrict__ pixtab,
                                                        float2 *__restrict__ U) {
    __shared__ float s_c[SKB][16];  // r1', r2', r3', -2 pi mu, a0, b0, g0, theta0
    __shared__ double s_f0[3];
    __shared__ int s_ref[2];
    const int tiles_x = (W + 63) / 64;
    const int tx = blockIdx.x % tiles_x, ty = blockIdx.x / tiles_x;
    const int l = blockIdx.y, k0 = blockIdx.z * SKB;
    const int nk = min(SKB, nb - k0);
    const int c_lo = tx * 64, r_lo = ty * 32;
    const double inv_lam = il.v[l];
    if (threadIdx.x == 0) {
        const int c_hi = min(c_lo + 64, W) - 1, r_hi = min(r_lo + 32, H) - 1;
        int c_ref, r_ref;
        tile_ref(c_lo, c_hi, r_lo, r_hi, H, W, dfx, dfy, inv_lam * inv_lam, c_ref, r_ref);
        const double f0x = (double)(c_ref - W / 2) * dfx, f0y = (double)(r_ref - H / 2) * dfy;
        s_f0[0] = f0x;
        s_f0[1] = f0y;
        s_f0[2] = sqrt(fmax(inv_lam * inv_lam - (f0x * f0x + f0y * f0y), 0.0));
        s_ref[0] = c_ref;
        s_ref[1] = r_ref;
    }
    __syncthreads();
    if (threadIdx.x < nk) {
        const int k = k0 + threadIdx.x;
        float *c = s_c[threadIdx.x];
        for (int m = 0; m < 9; ++m) c[m] = E.rr[9 * k + m];
        const double mu[3] = {E.mean[3 * k], E.mean[3 * k + 1], E.mean[3 * k + 2]};
        for (int m = 0; m < 3; ++m) c[9 + m] = (float)(-kTwoPi * mu[m]);
        const float fx = (float)s_f0[0], fy = (float)s_f0[1], fz = (float)s_f0[2], dz = (float)(s_f0[2] - inv_lam);
        c[12] = fmaf(c[2], dz, fmaf(c[1], fy, c[0] * fx));  // d = f - f_r at the reference
        c[13] = fmaf(c[5], dz, fmaf(c[4], fy, c[3] * fx));
        c[14] = fmaf(c[8], fz, fmaf(c[7], fy, c[6] * fx));
        double cyc = -(s_f0[0] * mu[0] + s_f0[1] * mu[1] + s_f0[2] * mu[2]);
        cyc -= rint(cyc);
        c[15] = (float)(kTwoPi * cyc);
    }
    __syncthreads();
    const long long hw = (long long)H * W;
    const bool even = ((H | W) & 1) == 0;
    const float2 *tab = pixtab + (size_t)l * hw;
    // pixel q = threadIdx.x + 256 p of the tile: a warp covers 32 consecutive columns of a row
#pragma unroll 2
    for (int p = 0; p < 8; ++p) {
        const int qq = threadIdx.x + 256 * p;
        const int row = r_lo + qq / 64, col = c_lo + qq % 64;
        if (row >= H || col >= W) continue;
        const size_t pix = (size_t)row * W + col;
        const float2 pt = tab[pix];
        const float dx = (float)((double)(col - s_ref[0]) * dfx), dy = (float)((double)(row - s_ref[1]) * dfy);
        float cs = 1.f, sn = 0.f;  // the centred-DFT pre-modulation e^{-j2pi(m r0/H + n c0/W)}
        if (even) {
            cs = ((row + col) & 1) ? -1.f : 1.f;
        } else {
            long long num = mod_num2(row, H / 2, 1, col, W / 2, 1, H, W);
            if (2 * num > hw) num -= hw;
            sincospif(-2.0f * (float)num / (float)hw, &sn, &cs);
        }
        for (int kk = 0; kk < nk; ++kk) {
            const float *c = s_c[kk];
            const float a = fmaf(c[2], pt.x, fmaf(c[1], dy, fmaf(c[0], dx, c[12])));
            const float b = fmaf(c[5], pt.x, fmaf(c[4], dy, fmaf(c[3], dx, c[13])));
            const float g = fmaf(c[8], pt.x, fmaf(c[7], dy, fmaf(c[6], dx, c[14])));
            const float t = fmaf(c[11], pt.x, fmaf(c[10], dy, fmaf(c[9], dx, c[15])));
            // |g| / f_z 2^-(a^2 + b^2) (pt.y = log2(1/f_z); -inf where evanescent)
            const float amp = fabsf(g) * ex2_approx(-fmaf(a, a, fmaf(b, b, -pt.y)));
            const float kr = __fadd_rn(fmaf(t, 0.15915494309189535f, 12582912.0f), -12582912.0f);
            const float ang = fmaf(kr, -6.28318530717958647692f, t);
            const float re = amp * cos_approx(ang), im = amp * sin_approx(ang);
            U[((size_t)(k0 + kk) * L + l) * hw + pix] = make_float2(re * cs - im * sn, re * sn + im * cs);
        }
    }
}

__global__ void k_fill(float *__restrict__ p, long long n, float v) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) p[i] = v;
}

// per pixel, in depth order over the batch: v_k = c_k o_k T u_k (in place), then T *= 1 - alpha_k
// uscale: the true field is uscale U (1 after the post-modulation; on even grids, where the post-
// and pre-modulations around the mask cancel to a constant, U is the raw inverse FFT and
// uscale = dfx dfy (-1)^(H/2 + W/2))
__global__ void k_exact_mask(float2 *__restrict__ U, float *__restrict__ Tm, ExactBatch E, int nb, int L, long long hw,
                             float t_eps, float t_bin, float uscale) {
    const long long pix = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const int l = blockIdx.y;
    if (pix >= hw) return;
    const long long idx = (long long)l * hw + pix;
    float T = Tm[idx];
    const float au = fabsf(uscale);
    const size_t kstride = (size_t)L * hw;
    float2 *base = U + idx;
    constexpr int KB = 8;  // fields loaded ahead of their masking (the loads do not wait on the stores)
    for (int k0 = 0; k0 < nb; k0 += KB) {
        float2 u[KB];
#pragma unroll
        for (int j = 0; j < KB; ++j)
            if (k0 + j < nb) u[j] = base[(size_t)(k0 + j) * kstride];
#pragma unroll
        for (int j = 0; j < KB; ++j) {
            const int k = k0 + j;
            if (k >= nb) break;
            const float sc = E.co[k * L + l] * T * uscale;
            base[(size_t)k * kstride] = make_float2(sc * u[j].x, sc * u[j].y);
            float a = E.ok[k] * au * sqrtf(u[j].x * u[j].x + u[j].y * u[j].y);
            if (!(a > t_eps)) a = 0.f;
            if (t_bin > 0.f) a = a > t_bin ? 1.f : 0.f;
            T *= 1.f - a;
        }
    }
    Tm[idx] = T;
}

constexpr int ETW = 64, ETH = 32, EPX = 8;  // the tiles of the per-pixel table (f_z - f0_z, log2 1/f_z)

// acc(f) += sum_k V_k(f) exp(-j 2 pi f_z z_k), f_z z_k = f0_z z_k (FP64, per tile) + (f_z - f0_z) z_k (FP32).
// FULL (partial coherence): the whole ramp exp(-j 2 pi f . mu_k) (x exp(+j 2 pi mu_z / lambda) with
// phase matching), anchored the same way: f . mu = f0 . mu (FP64) + (f - f0) . mu (FP32).
// V is the raw forward FFT times vscale, and with fold also times (-1)^(r + c) (the even-grid
// post-modulation folded in); otherwise the already post-modulated spectrum (vscale = 1).
template <bool FULL>
__global__ void __launch_bounds__((ETW / EPX) * ETH) k_exact_accum(const float2 *__restrict__ V, float2 *__restrict__ acc,
                                                                   const float2 *__restrict__ pixtab, ExactBatch E,
                                                                   int nb, int L, int H, int W, double dfx, double dfy,
                                                                   InvLam il, int phase_match, int fold, float vscale) {
    __shared__ float s_th[GWS_MAX_SCENES], s_mz[GWS_MAX_SCENES], s_mx[GWS_MAX_SCENES], s_my[GWS_MAX_SCENES];
    __shared__ double s_f0z, s_f0x, s_f0y;
    __shared__ int s_cref, s_rref;
    const int tiles_x = (W + ETW - 1) / ETW;
    const int tx = blockIdx.x % tiles_x, ty = blockIdx.x / tiles_x;
    const int l = blockIdx.y;
    const int c_lo = tx * ETW, r_lo = ty * ETH;
    const double inv_lam = il.v[l];
    if (threadIdx.x == 0) {
        const int c_hi = min(c_lo + ETW, W) - 1, r_hi = min(r_lo + ETH, H) - 1;
        int c_ref, r_ref;
        tile_ref(c_lo, c_hi, r_lo, r_hi, H, W, dfx, dfy, inv_lam * inv_lam, c_ref, r_ref);
        const double f0x = (double)(c_ref - W / 2) * dfx, f0y = (double)(r_ref - H / 2) * dfy;
        s_f0z = sqrt(fmax(inv_lam * inv_lam - (f0x * f0x + f0y * f0y), 0.0));
        s_f0x = f0x;
        s_f0y = f0y;
        s_cref = c_ref;
        s_rref = r_ref;
    }
    __syncthreads();
    for (int k = threadIdx.x; k < nb; k += blockDim.x) {
        if (FULL) {
            const double mx = E.mu[3 * k], my = E.mu[3 * k + 1], mz = E.mu[3 * k + 2];
            double cyc = -(s_f0x * mx + s_f0y * my + s_f0z * mz);
            if (phase_match) cyc += mz * inv_lam;
            cyc -= rint(cyc);
            s_th[k] = (float)(kTwoPi * cyc);
            s_mx[k] = (float)(-kTwoPi * mx);
            s_my[k] = (float)(-kTwoPi * my);
            s_mz[k] = (float)(-kTwoPi * mz);
        } else {
            double cyc = -s_f0z * E.zk[k];
            cyc -= rint(cyc);
            s_th[k] = (float)(kTwoPi * cyc);
            s_mz[k] = (float)(-kTwoPi * E.zk[k]);
        }
    }
    __syncthreads();
    const long long hw = (long long)H * W;
    // pixel q = threadIdx.x + 256 p of the tile: a warp covers 32 consecutive columns of a row
#pragma unroll
    for (int p = 0; p < EPX; ++p) {
        const int q = threadIdx.x + (ETW / EPX) * ETH * p;
        const int row = r_lo + q / ETW, col = c_lo + q % ETW;
        if (row >= H || col >= W) continue;
        const float dyf = (float)((double)(row - s_rref) * dfy);
        const long long pix = (long long)row * W + col;
        const float2 pt = pixtab[(size_t)l * hw + pix];
        if (!(pt.y > -INFINITY)) continue;  // evanescent: H = 0
        const float dxf = (float)((double)(col - s_cref) * dfx);
        float2 a = make_float2(0.f, 0.f);
        for (int k = 0; k < nb; ++k) {
            const float2 v = V[((size_t)k * L + l) * hw + pix];
            const float t = FULL ? fmaf(s_mz[k], pt.x, fmaf(s_my[k], dyf, fmaf(s_mx[k], dxf, s_th[k])))
                                 : fmaf(s_mz[k], pt.x, s_th[k]);
            const float kr = __fadd_rn(fmaf(t, 0.15915494309189535f, 12582912.0f), -12582912.0f);
            const float ang = fmaf(kr, -6.28318530717958647692f, t);
            float sn, cs;
            __sincosf(ang, &sn, &cs);
            a.x = fmaf(v.x, cs, fmaf(-v.y, sn, a.x));
            a.y = fmaf(v.x, sn, fmaf(v.y, cs, a.y));
        }
        const float sg = (fold && ((row + col) & 1)) ? -vscale : vscale;
        float2 cur = acc[(size_t)l * hw + pix];
        cur.x = fmaf(sg, a.x, cur.x);
        cur.y = fmaf(sg, a.y, cur.y);
        acc[(size_t)l * hw + pix] = cur;
    }
}

// ---- partial coherence (Eq. 14) ---------------------------------------------------------

// SplitMix64 (Steele, Lea and Flood, 2014): output number `ctr` of the stream seeded with `seed`
__device__ __forceinline__ unsigned long long splitmix64(unsigned long long seed, unsigned long long ctr) {
    unsigned long long z = seed + ctr * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// real spherical harmonic Y_l^m (degree <= 3, Condon-Shortley phase, normalised) at unit (x, y, z)
__device__ double sh_lm(int l, int m, double x, double y, double z) {
    const double pi = 3.14159265358979323846;
    switch (l * l + l + m) {
        case 0: return 0.5 / sqrt(pi);
        case 1: return -sqrt(3.0 / (4.0 * pi)) * y;
        case 2: return sqrt(3.0 / (4.0 * pi)) * z;
        case 3: return -sqrt(3.0 / (4.0 * pi)) * x;
        case 4: return sqrt(15.0 / (4.0 * pi)) * x * y;
        case 5: return -sqrt(15.0 / (4.0 * pi)) * y * z;
        case 6: return sqrt(5.0 / (16.0 * pi)) * (3.0 * z * z - 1.0);
        case 7: return -sqrt(15.0 / (4.0 * pi)) * x * z;
        case 8: return sqrt(15.0 / (16.0 * pi)) * (x * x - y * y);
        case 9: return -sqrt(35.0 / (32.0 * pi)) * y * (3.0 * x * x - y * y);
        case 10: return sqrt(105.0 / (4.0 * pi)) * x * y * z;
        case 11: return -sqrt(21.0 / (32.0 * pi)) * y * (5.0 * z * z - 1.0);
        case 12: return sqrt(7.0 / (16.0 * pi)) * z * (5.0 * z * z - 3.0);
        case 13: return -sqrt(21.0 / (32.0 * pi)) * x * (5.0 * z * z - 1.0);
        case 14: return sqrt(105.0 / (16.0 * pi)) * z * (x * x - y * y);
        default: return -sqrt(35.0 / (32.0 * pi)) * x * (x * x - 3.0 * y * y);
    }
}

// K(f) = Y_l^m(lambda f) e^{j phi(f)} on the centred grid (0 where evanescent); ysum[l] += sum Y^2
__global__ void __launch_bounds__(256) k_pc_kernel(float2 *__restrict__ K, double *__restrict__ ysum, int sh_l, int sh_m,
                                                   unsigned long long seed, unsigned long long frame, int L, int H,
                                                   int W, double dfx, double dfy, InvLam il) {
    __shared__ double red[8];
    const long long hw = (long long)H * W;
    const int l = blockIdx.y;
    const long long pix = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    double y2 = 0.0;
    if (pix < hw) {
        const int r = (int)(pix / W), c = (int)(pix % W);
        const double lam = 1.0 / il.v[l];
        const double fx = (double)(c - W / 2) * dfx, fy = (double)(r - H / 2) * dfy;
        const double k2 = il.v[l] * il.v[l], rho2 = fx * fx + fy * fy;
        float2 v = make_float2(0.f, 0.f);
        if (rho2 < k2) {
            const double fz = sqrt(k2 - rho2);
            const double Y = sh_lm(sh_l, sh_m, fx * lam, fy * lam, fz * lam);
            const unsigned long long ctr = (frame * (unsigned long long)L + (unsigned long long)l) * (unsigned long long)hw +
                                           (unsigned long long)pix + 1ull;
            const double u = (double)(splitmix64(seed, ctr) >> 11) * 0x1.0p-53;
            double sn, cs;
            sincos(6.283185307179586476925 * u - 3.14159265358979323846, &sn, &cs);
            v = make_float2((float)(Y * cs), (float)(Y * sn));
            y2 = Y * Y;
        }
        K[(size_t)l * hw + pix] = v;
    }
    for (int o = 16; o > 0; o >>= 1) y2 += __shfl_xor_sync(0xffffffffu, y2, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = y2;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
        atomicAdd(ysum + l, t);
    }
}

// grid (pixel blocks, k L + l): no index division per value
__global__ void k_pc_apply(const float2 *Uin, float2 *Uout, const float2 *__restrict__ kappa,
                           const double *__restrict__ ysum, ExactBatch E, int nb, int L, long long hw, float uscale) {
    __shared__ float s_s;
    const int kl = blockIdx.y;  // k * L + l
    const int l = kl % L;
    if (threadIdx.x == 0) s_s = E.co[kl] * uscale * (float)(1.0 / sqrt(ysum[l]));  // FP64 once per block
    __syncthreads();
    const long long pix = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (pix >= hw) return;
    const float s = s_s;
    const float2 a = kappa[(size_t)l * hw + pix];
    const size_t idx = (size_t)kl * hw + pix;
    const float2 u = Uin[idx];
    Uout[idx] = make_float2(s * (u.x * a.x - u.y * a.y), s * (u.x * a.y + u.y * a.x));
}

static inline unsigned nblk(long long n, int t) { return (unsigned)((n + t - 1) / t); }

cudaError_t launch_exact_gather(const unsigned *sorted, long long b0, int nb, const gws_gaussians *g, int L,
                                const ExactBatch &E, int pc, cudaStream_t s) {
    k_exact_gather<<<nblk(nb, 128), 128, 0, s>>>(sorted, b0, nb, g->mean, g->quat, g->scale, g->opacity, g->amp, L, E,
                                                 pc);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_fill(float *p, long long n, float v, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    k_fill<<<nblk(n, 256), 256, 0, s>>>(p, n, v);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_single_spectra(const ExactBatch &E, int nb, int L, int H, int W, double dfx, double dfy,
                                  const InvLam &il, const float2 *pixtab, float2 *U, cudaStream_t s) {
    const int tiles = ((W + 63) / 64) * ((H + 31) / 32);
    k_single_spectra<<<dim3(tiles, L, (nb + SKB - 1) / SKB), 256, 0, s>>>(E, nb, L, H, W, dfx, dfy, il, pixtab, U);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_exact_mask(float2 *U, float *T, const ExactBatch &E, int nb, int L, long long hw, float t_eps,
                              float t_bin, float uscale, cudaStream_t s) {
    k_exact_mask<<<dim3(nblk(hw, 256), (unsigned)L), 256, 0, s>>>(U, T, E, nb, L, hw, t_eps, t_bin, uscale);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_exact_accum(const float2 *V, float2 *acc, const float2 *pixtab, const ExactBatch &E, int nb, int L,
                               int H, int W, double dfx, double dfy, const InvLam &il, int fold, float vscale,
                               cudaStream_t s) {
    const int tiles = ((W + ETW - 1) / ETW) * ((H + ETH - 1) / ETH);
    k_exact_accum<false><<<dim3(tiles, L), (ETW / EPX) * ETH, 0, s>>>(V, acc, pixtab, E, nb, L, H, W, dfx, dfy, il, 0,
                                                                      fold, vscale);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_pc_kernel(float2 *K, double *ysum, int sh_l, int sh_m, unsigned long long seed,
                             unsigned long long frame, int L, int H, int W, double dfx, double dfy, const InvLam &il,
                             cudaStream_t s) {
    const long long hw = (long long)H * W;
    k_pc_kernel<<<dim3(nblk(hw, 256), L), 256, 0, s>>>(K, ysum, sh_l, sh_m, seed, frame, L, H, W, dfx, dfy, il);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_pc_apply(const float2 *Uin, float2 *Uout, const float2 *kappa, const double *ysum,
                            const ExactBatch &E, int nb, int L, long long hw, float uscale, cudaStream_t s) {
    k_pc_apply<<<dim3(nblk(hw, 256), nb * L), 256, 0, s>>>(Uin, Uout, kappa, ysum, E, nb, L, hw, uscale);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_pc_accum(const float2 *V, float2 *acc, const float2 *pixtab, const ExactBatch &E, int nb, int L,
                            int H, int W, double dfx, double dfy, const InvLam &il, int phase_match, int fold,
                            float vscale, cudaStream_t s) {
    const int tiles = ((W + ETW - 1) / ETW) * ((H + ETH - 1) / ETH);
    k_exact_accum<true><<<dim3(tiles, L), (ETW / EPX) * ETH, 0, s>>>(V, acc, pixtab, E, nb, L, H, W, dfx, dfy, il,
                                                                     phase_match, fold, vscale);
    count_launches(1);
    return cudaGetLastError();
}

}  // namespace gws
