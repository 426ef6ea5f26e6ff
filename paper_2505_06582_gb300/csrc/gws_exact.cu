// gws_exact.cu -- exact alpha wave blending (Eq. 5-6 with the spatial transmittance map,
// Algorithm S2), front to back over depth-ordered batches of Gaussians:
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
                               const float *__restrict__ opacity, const float *__restrict__ amp, int L, ExactBatch E) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= nb) return;
    const long long i = sorted[b0 + k];
    E.mean[3 * k] = mean[3 * i];
    E.mean[3 * k + 1] = mean[3 * i + 1];
    E.mean[3 * k + 2] = 0.0;  // the field on the Gaussian's own plane
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

__global__ void k_fill(float *__restrict__ p, long long n, float v) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) p[i] = v;
}

// per pixel, in depth order over the batch: v_k = c_k o_k T u_k (in place), then T *= 1 - alpha_k
__global__ void k_exact_mask(float2 *__restrict__ U, float *__restrict__ Tm, ExactBatch E, int nb, int L, long long hw,
                             float t_eps, float t_bin) {
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= hw * L) return;
    const int l = (int)(idx / hw);
    const long long pix = idx % hw;
    float T = Tm[idx];
    for (int k = 0; k < nb; ++k) {
        float2 *up = U + ((size_t)k * L + l) * hw + pix;
        const float2 u = *up;
        const float s = E.co[k * L + l] * T;
        *up = make_float2(s * u.x, s * u.y);
        float a = E.ok[k] * sqrtf(u.x * u.x + u.y * u.y);
        if (!(a > t_eps)) a = 0.f;
        if (t_bin > 0.f) a = a > t_bin ? 1.f : 0.f;
        T *= 1.f - a;
    }
    Tm[idx] = T;
}

constexpr int ETW = 64, ETH = 32, EPX = 8;  // the tiles of the per-pixel table (f_z - f0_z, log2 1/f_z)

// acc(f) += sum_k V_k(f) exp(-j 2 pi f_z z_k), f_z z_k = f0_z z_k (FP64, per tile) + (f_z - f0_z) z_k (FP32)
__global__ void __launch_bounds__((ETW / EPX) * ETH) k_exact_accum(const float2 *__restrict__ V, float2 *__restrict__ acc,
                                                                   const float2 *__restrict__ pixtab, ExactBatch E,
                                                                   int nb, int L, int H, int W, double dfx, double dfy,
                                                                   InvLam il) {
    __shared__ float s_th[GWS_MAX_SCENES], s_mz[GWS_MAX_SCENES];
    __shared__ double s_f0z;
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
    }
    __syncthreads();
    for (int k = threadIdx.x; k < nb; k += blockDim.x) {
        double cyc = -s_f0z * E.zk[k];
        cyc -= rint(cyc);
        s_th[k] = (float)(kTwoPi * cyc);
        s_mz[k] = (float)(-kTwoPi * E.zk[k]);
    }
    __syncthreads();
    const int row = r_lo + threadIdx.x / (ETW / EPX);
    const int col0 = c_lo + (threadIdx.x % (ETW / EPX)) * EPX;
    if (row >= H) return;
    const long long hw = (long long)H * W;
#pragma unroll
    for (int p = 0; p < EPX; ++p) {
        const int col = col0 + p;
        if (col >= W) break;
        const long long pix = (long long)row * W + col;
        const float2 pt = pixtab[(size_t)l * hw + pix];
        if (!(pt.y > -INFINITY)) continue;  // evanescent: H = 0
        float2 a = acc[(size_t)l * hw + pix];
        for (int k = 0; k < nb; ++k) {
            const float2 v = V[((size_t)k * L + l) * hw + pix];
            const float t = fmaf(s_mz[k], pt.x, s_th[k]);
            const float kr = __fadd_rn(fmaf(t, 0.15915494309189535f, 12582912.0f), -12582912.0f);
            const float ang = fmaf(kr, -6.28318530717958647692f, t);
            float sn, cs;
            __sincosf(ang, &sn, &cs);
            a.x = fmaf(v.x, cs, fmaf(-v.y, sn, a.x));
            a.y = fmaf(v.x, sn, fmaf(v.y, cs, a.y));
        }
        acc[(size_t)l * hw + pix] = a;
    }
}

static inline unsigned nblk(long long n, int t) { return (unsigned)((n + t - 1) / t); }

cudaError_t launch_exact_gather(const unsigned *sorted, long long b0, int nb, const gws_gaussians *g, int L,
                                const ExactBatch &E, cudaStream_t s) {
    k_exact_gather<<<nblk(nb, 128), 128, 0, s>>>(sorted, b0, nb, g->mean, g->quat, g->scale, g->opacity, g->amp, L, E);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_fill(float *p, long long n, float v, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    k_fill<<<nblk(n, 256), 256, 0, s>>>(p, n, v);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_exact_mask(float2 *U, float *T, const ExactBatch &E, int nb, int L, long long hw, float t_eps,
                              float t_bin, cudaStream_t s) {
    k_exact_mask<<<nblk(hw * L, 256), 256, 0, s>>>(U, T, E, nb, L, hw, t_eps, t_bin);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_exact_accum(const float2 *V, float2 *acc, const float2 *pixtab, const ExactBatch &E, int nb, int L,
                               int H, int W, double dfx, double dfy, const InvLam &il, cudaStream_t s) {
    const int tiles = ((W + ETW - 1) / ETW) * ((H + ETH - 1) / ETH);
    k_exact_accum<<<dim3(tiles, L), (ETW / EPX) * ETH, 0, s>>>(V, acc, pixtab, E, nb, L, H, W, dfx, dfy, il);
    count_launches(1);
    return cudaGetLastError();
}

}  // namespace gws
