// gws_common.cuh -- internal types and device helpers of libgws (sm_103a).
//
// Notation follows the paper (arXiv 2505.06582): a Gaussian has mean mu, rotation
// columns r1 (t_u), r2 (t_v), r3 (normal), scales s_u, s_v, opacity o and amplitude c per
// wavelength (Sec. 3).  Its spectrum at the SLM is Eq. 10 with the reference-wave shift
// (Sec. 4.1); spectra are summed by Eq. 12 (or Eq. 5-6 with T at the centre).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/gws.h"

namespace gws {

constexpr double kPi = 3.14159265358979323846;
constexpr double kTwoPi = 6.28318530717958647692;
// exp(-2 pi^2 x) = 2^(-x * 2 pi^2 / ln 2): kappa = pi * sqrt(2 / ln 2) folds the 2 pi^2 and
// the base change into the scaled rotation columns, so the per-pair exponent is an ex2.
constexpr double kKappa = 5.336446256636997;  // pi * sqrt(2 / ln 2)

// Device status bits (a word in the workspace; the host maps them to gws_status).
enum : int {
    ST_NONFINITE = 1,
    ST_BADVALUE = 2,
    ST_TIMEOUT = 4,
    ST_BOUNDS = 8,  // bounds-checking build: an index out of range (access skipped) or a canary overwritten
};

// Bounds checks of the checking build (GWS_CHECK_BOUNDS): in_bounds(ok, status) records a failed
// check in the status word and returns ok, so that the caller skips the access; the product
// build compiles every check to `true`.
#ifdef GWS_CHECK_BOUNDS
__device__ __forceinline__ bool in_bounds(bool ok, int *status) {
    if (!ok && status) atomicOr(status, ST_BOUNDS);
    return ok;
}
#else
__device__ __forceinline__ constexpr bool in_bounds(bool, int *) { return true; }
#endif

// Per-Gaussian data after validation (concatenated over scenes, input order).
struct alignas(16) GPre {
    double mu[3];
    double q[4];  // normalised quaternion (w, x, y, z)
    float su, sv, o;
    int scene;
};

// One Gaussian's record for one wavelength, as the splat kernels stream it (96 bytes, a
// multiple of 16 so that 1-D bulk copies of whole chunks stay 16-byte aligned).
//   r1' = kappa s_u r1, r2' = kappa s_v r2 (so that 2^-(a'^2 + b'^2) is the Gaussian factor),
//   r3' = W r3 (forward) or r3 (backward), W = 2 pi s_u s_v c o T (Eq. 10 amplitude x Eq. 12 weight),
//   m = -2 pi mu in FP32 for the in-tile phase deltas (radians), mu in FP64 for the per-tile
//   phase anchor,
//   e = footprint ellipse normalised to 1.
struct alignas(16) Rec {
    float r1x, r1y, r1z, r2x;
    float r2y, r2z, r3x, r3y;
    float r3z, mx, my, mz;
    float e00, e01, e11, W;
    double mux, muy;
    double muz;
    int g;     // global (concatenated) Gaussian index
    float wz;  // |(s_u r1z, s_v r2z)| / rho': how fast the footprint shrinks with the tile's bound on |d_z|
};
static_assert(sizeof(Rec) == 96, "record must stay 96 bytes");

// Per depth-sorted Gaussian data of the transmittance pass (FP64 like the oracle).
struct alignas(16) TData {
    double mx, my;
    double m00, m01, m10, m11, det;
    float o;
    float bx0, bx1, by0, by1;  // box outside which alpha < alpha_min
    float pad;
};

// Per depth-sorted Gaussian: the product of its non-unit front factors (1 - alpha) and the
// number of factors equal to 0 (alpha = 1), so that T = n1 ? 0 : Tnz, and dL/dT.
struct alignas(16) TQuery {
    double Tnz;
    double dT;
    int n1;
    int pad;
};

// FP64 path record (per depth-sorted Gaussian).
struct alignas(16) Rec64 {
    double r1[3], r2[3], r3[3];
    double mu[3];
    double su, sv;
};

struct SceneTable {
    int n_scenes;
    int n_lambda;
    long long off[GWS_MAX_SCENES + 1];
    const double *mean[GWS_MAX_SCENES];
    const float *quat[GWS_MAX_SCENES];
    const float *scale[GWS_MAX_SCENES];
    const float *opacity[GWS_MAX_SCENES];
    const float *amp[GWS_MAX_SCENES];
};

struct Grid {
    int H, W;
    double px, py;
    int n_lambda;
    double lam[GWS_MAX_LAMBDA];
};

// ---------------------------------------------------------------------------------------
// device helpers
// ---------------------------------------------------------------------------------------

__device__ __forceinline__ int scene_of(const long long *off, int n_scenes, long long g) {
    int lo = 0, hi = n_scenes - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (off[mid] <= g) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// Rotation columns of a normalised quaternion (w, x, y, z).
template <typename T>
__device__ __forceinline__ void quat_cols(const T q[4], T r1[3], T r2[3], T r3[3]) {
    T w = q[0], x = q[1], y = q[2], z = q[3];
    r1[0] = T(1) - T(2) * (y * y + z * z);
    r1[1] = T(2) * (x * y + w * z);
    r1[2] = T(2) * (x * z - w * y);
    r2[0] = T(2) * (x * y - w * z);
    r2[1] = T(1) - T(2) * (x * x + z * z);
    r2[2] = T(2) * (y * z + w * x);
    r3[0] = T(2) * (x * z + w * y);
    r3[1] = T(2) * (y * z - w * x);
    r3[2] = T(1) - T(2) * (x * x + y * y);
}

// packed f32x2 helpers: both lanes of a pair equal; sign(g) e for e >= 0 (g's sign bit on e)
__device__ __forceinline__ float2 pair(float x) { return make_float2(x, x); }
__device__ __forceinline__ float2 neg2(float2 x) { return make_float2(-x.x, -x.y); }
__device__ __forceinline__ float with_sign_of(float e, float g) {
    return __int_as_float(__float_as_int(e) ^ (__float_as_int(g) & 0x80000000));
}

__device__ __forceinline__ float ex2_approx(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float sin_approx(float x) {
    float y;
    asm("sin.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float cos_approx(float x) {
    float y;
    asm("cos.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// ---- mbarrier + 1-D bulk copy (TMA engine) -------------------------------------------

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void fence_proxy_async() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// Bounded wait: returns false if the phase did not complete within `limit` cycles.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity, unsigned long long limit) {
    if (mbar_try_wait(bar, parity)) return true;
    unsigned long long t0 = clock64();
    while (true) {
        if (mbar_try_wait(bar, parity)) return true;
        if (clock64() - t0 > limit) return false;
    }
}
// global -> shared bulk copy, completion counted on `bar` (bytes multiple of 16, both
// addresses 16-byte aligned).
__device__ __forceinline__ void bulk_g2s(void *smem_dst, const void *gmem_src, uint32_t bytes, uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(smem_dst)),
        "l"(gmem_src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

// Reference frequency of a tile: the centre of its valid pixels, or -- when that is
// evanescent -- its pixel nearest to f = 0, so that |f - f0| stays within the tile.
__host__ __device__ __forceinline__ void tile_ref(int c_lo, int c_hi, int r_lo, int r_hi, int H, int W, double dfx,
                                                  double dfy, double k2, int &c_ref, int &r_ref) {
    c_ref = (c_lo + c_hi + 1) / 2;
    r_ref = (r_lo + r_hi + 1) / 2;
    const double fx = (double)(c_ref - W / 2) * dfx, fy = (double)(r_ref - H / 2) * dfy;
    if (fx * fx + fy * fy >= k2) {
        c_ref = W / 2 < c_lo ? c_lo : (W / 2 > c_hi ? c_hi : W / 2);
        r_ref = H / 2 < r_lo ? r_lo : (H / 2 > r_hi ? r_hi : H / 2);
    }
}

// Range [fzlo, fzhi] of f_z = sqrt(1/lambda^2 - f_x^2 - f_y^2) over the frequency rectangle
// [x0, x1] x [y0, y1] (FP64): its points nearest to and farthest from f = 0 (0 where evanescent).
__host__ __device__ __forceinline__ void fz_range(double x0, double x1, double y0, double y1, double k2, float &fzlo,
                                                  float &fzhi) {
    const double nx = x0 > 0.0 ? x0 : (x1 < 0.0 ? x1 : 0.0), ny = y0 > 0.0 ? y0 : (y1 < 0.0 ? y1 : 0.0);
    const double fx = fmax(fabs(x0), fabs(x1)), fy = fmax(fabs(y0), fabs(y1));
    fzhi = (float)sqrt(fmax(k2 - (nx * nx + ny * ny), 0.0));
    fzlo = (float)sqrt(fmax(k2 - (fx * fx + fy * fy), 0.0));
}

// The sign of g = r3.f over the box [x0, x1] x [y0, y1] x [fzlo, fzhi] when it is the same at
// every point (+1 / -1), else 0: g is linear in f, so its bounds are sums of per-axis extremes;
// a margin of 1e-5 of its terms covers the FP32 evaluation of g at a pixel.
__device__ __forceinline__ int sign_over_box(float r3x, float r3y, float r3z, float x0, float x1, float y0, float y1,
                                             float fzlo, float fzhi) {
    const float lo = fminf(r3x * x0, r3x * x1) + fminf(r3y * y0, r3y * y1) + fminf(r3z * fzlo, r3z * fzhi);
    const float hi = fmaxf(r3x * x0, r3x * x1) + fmaxf(r3y * y0, r3y * y1) + fmaxf(r3z * fzlo, r3z * fzhi);
    const float tol = 1e-5f * (fabsf(r3x) * fmaxf(fabsf(x0), fabsf(x1)) + fabsf(r3y) * fmaxf(fabsf(y0), fabsf(y1)) +
                               fabsf(r3z) * fzhi);
    return lo > tol ? 1 : (hi < -tol ? -1 : 0);
}

// The largest |f_z - 1/lambda| over the frequency rectangle [x0, x1] x [y0, y1]: at its point
// farthest from f = 0 (1/lambda where that point is evanescent).
__host__ __device__ __forceinline__ double dz_far(double x0, double x1, double y0, double y1, double inv_lam) {
    const double fx = fmax(fabs(x0), fabs(x1)), fy = fmax(fabs(y0), fabs(y1));
    return inv_lam - sqrt(fmax(inv_lam * inv_lam - (fx * fx + fy * fy), 0.0));
}

// The footprint ellipse of a record over a tile whose |d_z| stays within dzt, from the grid-wide
// one (built for |d_z| <= dzmax): rho' shrinks to rho + dzt |(s_u r1z, s_v r2z)|, i.e. by the factor
// rt = 1 - (dzmax - dzt) wz, and the ellipse's matrix grows by 1 / rt^2.
__device__ __forceinline__ float footprint_scale(float dzmax, float dzt, float wz) {
    const float rt = 1.f - fmaxf(dzmax - dzt, 0.f) * wz;
    return 1.f / (rt * rt);
}

// Centred-DFT modulation angle, in cycles: ((a * b) mod n) / n, exact integer reduction.
__device__ __forceinline__ double mod_frac(long long a, long long b, long long n) {
    long long m = (a * b) % n;
    if (m < 0) m += n;
    return (double)m / (double)n;
}

// The same angles combined over both axes as one integer numerator of the denominator H W:
//   (sh * ((a * b) mod H) * W + sw * ((c * d) mod W) * H) mod (H W),  sh, sw in {-1, +1};
// the angle in cycles is num / (H W) (exact integers; one multiply by 1/(H W) afterwards).
__device__ __forceinline__ long long mod_num2(long long a, long long b, int sh, long long c, long long d, int sw,
                                              long long H, long long W) {
    long long mh = (a * b) % H, mw = (c * d) % W;
    if (mh < 0) mh += H;
    if (mw < 0) mw += W;
    long long num = (sh * mh * W + sw * mw * H) % (H * W);
    return num < 0 ? num + H * W : num;
}

}  // namespace gws
