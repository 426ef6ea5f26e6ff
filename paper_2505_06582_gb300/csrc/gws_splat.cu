// gws_splat.cu -- forward splat: u_SLM(f) = sum_i W_i |r3.f|/f_z exp(-2 pi^2 [..]) exp(-j 2 pi f.mu_i)
// (Eq. 10 summed by Eq. 12, or by Eq. 5-6 with T_i at the centre; the weights arrive in W).
//
// Mixed-precision persistent tile splat.  A work item is one (scene, wavelength, frequency
// tile).  A CTA holds the tile's complex accumulators in registers (PX consecutive pixels
// of one row per thread) and streams the segment's Gaussian records through shared
// memory with 1-D bulk copies (cp.async.bulk, mbarrier completion, STAGES-deep ring of
// one-record-per-thread chunks).
// Records are ordered by decreasing spectral footprint radius, so a tile only reads the
// prefix of records whose footprint can reach it (item_count); an exact ellipse-rectangle
// test then culls per (record, tile).
//
// Precision: the phase -f.mu reaches ~2e4 cycles.  Per (record, tile) it is split into an
// FP64 anchor at the tile's reference frequency f0, reduced mod 1 in FP64, plus FP32
// deltas (f - f0).mu inside the tile (|.| < ~20 cycles); per (record, thread) the FP32 phase at
// the thread's middle column is reduced to [-pi, pi], and the pixels' phases (a few cycles
// from it) go to sin/cos unreduced (the record carries -2 pi mu, the anchor is in radians).  f0 is
// the centre of the tile's valid pixels; f_z and f_z - f0_z are formed in FP64 once per pixel
// and item, and 1/f_z enters as log2(1/f_z) inside the exponent.  Per-chunk FP32 sums are
// merged into a TwoSum-compensated FP32 total.
#include "gws_host.h"

namespace gws {

// Smallest value of the quadratic form f^T E f over the rectangle [x0,x1] x [y0,y1] is <= 1?
__device__ __forceinline__ bool ellipse_hits_rect(float e00, float e01, float e11, float x0, float x1, float y0,
                                                  float y1) {
    if (x0 <= 0.f && 0.f <= x1 && y0 <= 0.f && 0.f <= y1) return true;
    float best = 3.0e38f;
    // vertical edges x = xe, y in [y0, y1]
#pragma unroll
    for (int k = 0; k < 2; ++k) {
        float xe = k ? x1 : x0;
        float ys = e11 > 0.f ? fminf(fmaxf(-e01 * xe / e11, y0), y1) : y0;
        best = fminf(best, e00 * xe * xe + 2.f * e01 * xe * ys + e11 * ys * ys);
    }
#pragma unroll
    for (int k = 0; k < 2; ++k) {
        float ye = k ? y1 : y0;
        float xs = e00 > 0.f ? fminf(fmaxf(-e01 * ye / e00, x0), x1) : x0;
        best = fminf(best, e00 * xs * xs + 2.f * e01 * xs * ye + e11 * ye * ye);
    }
    return best <= 1.001f;
}

__device__ __forceinline__ void two_sum_acc(float &s, float &c, float x) {
    float t = s + x;
    float bp = t - s;
    c += (s - (t - bp)) + (x - bp);
    s = t;
}

// cos of a phase within a few turns of zero on the FP32 pipe (both lanes of a pair): the nearest
// whole turn is taken off with a two-part 2 pi (float(2 pi) and its remainder), then an even
// degree-12 polynomial in r^2 gives cos(r), |r| <= pi.  The coefficients were fitted for this
// kernel to cos on [-pi, pi] (least squares reweighted toward the minimax error; |error| of the
// FP32 evaluation <= 4.4e-7, below sin/cos.approx's on the unreduced arguments).  It moves part of
// the MUFU's load onto the FMA pipe.
__device__ __forceinline__ float2 cos_poly2(float2 x) {
    const float2 k = __fadd2_rn(__ffma2_rn(x, pair(0.15915494309189535f), pair(12582912.0f)), pair(-12582912.0f));
    float2 r = __ffma2_rn(k, pair(-6.28318548202514648f), x);
    r = __ffma2_rn(k, pair(1.74845553e-7f), r);
    const float2 t = __fmul2_rn(r, r);
    float2 p = __ffma2_rn(t, pair(1.7244632e-09f), pair(-2.7078977e-07f));
    p = __ffma2_rn(p, t, pair(2.4769886e-05f));
    p = __ffma2_rn(p, t, pair(-1.3887804e-03f));
    p = __ffma2_rn(p, t, pair(4.1666489e-02f));
    p = __ffma2_rn(p, t, pair(-4.9999988e-01f));
    return __ffma2_rn(p, t, pair(1.0f));
}

// One listed record over this thread's PH pixel pairs (packed f32x2): the Gaussian factor and
// the phase of Eq. 10 from the per-(record, tile) scalars sv[0..3], accumulated into acc.  The
// linear forms are anchored at the thread's middle column (offset dxm from the tile's reference
// frequency; the pixels sit at ddx from it), and the phase there is reduced to [-pi, pi] once per
// record, so the per-pixel phase stays within |t_x ddx| + |t_z dz| + pi of zero and goes to
// sin/cos unreduced (the argument error of sin.approx grows like 1.2e-7 |t|).  The cos of the
// first NPOLY pairs runs on the FP32 pipe (cos_poly2) instead of the MUFU.
template <int PH, int NPOLY>
__device__ __forceinline__ void splat_record(const float4 *__restrict__ sv, float dy, float dxm, const float2 *ddx,
                                             const float2 *dz, const float2 *lfz, float2 *acc_re, float2 *acc_im) {
    const float4 Ar = sv[0], Br = sv[1], Gr = sv[2], Mr = sv[3];
    const float2 ar = pair(fmaf(Ar.x, dxm, fmaf(Ar.y, dy, Ar.w))), br = pair(fmaf(Br.x, dxm, fmaf(Br.y, dy, Br.w)));
    const float2 gr = pair(fmaf(Gr.x, dxm, fmaf(Gr.y, dy, Gr.w)));
    // t (radians) at the middle column minus 2 pi round(t / 2 pi), rounding on the FP32 pipe (+-1.5 * 2^23)
    const float t0 = fmaf(Mr.x, dxm, fmaf(Mr.y, dy, Mr.w));
    const float k0 = __fadd_rn(fmaf(t0, 0.15915494309189535f, 12582912.0f), -12582912.0f);
    const float2 tr = pair(fmaf(k0, -6.28318530717958647692f, t0));
    const float2 ax = pair(Ar.x), az = pair(Ar.z), bx = pair(Br.x), bz = pair(Br.z);
    const float2 gx = pair(Gr.x), gz = pair(Gr.z), tx2 = pair(Mr.x), tz = pair(Mr.z);
#pragma unroll
    for (int h = 0; h < PH; ++h) {
        const float2 a = __ffma2_rn(az, dz[h], __ffma2_rn(ax, ddx[h], ar));
        const float2 b = __ffma2_rn(bz, dz[h], __ffma2_rn(bx, ddx[h], br));
        const float2 g = __ffma2_rn(gz, dz[h], __ffma2_rn(gx, ddx[h], gr));
        const float2 ang = __ffma2_rn(tz, dz[h], __ffma2_rn(tx2, ddx[h], tr));
        // |g| / f_z 2^-(a^2 + b^2) = g (sign(g) 2^-(a^2 + b^2 + log2 f_z))
        const float2 u = __ffma2_rn(a, a, __ffma2_rn(b, b, lfz[h]));
        const float2 amp = __fmul2_rn(g, make_float2(with_sign_of(ex2_approx(-u.x), g.x),
                                                     with_sign_of(ex2_approx(-u.y), g.y)));
        const float2 cs = h < NPOLY ? cos_poly2(ang) : make_float2(cos_approx(ang.x), cos_approx(ang.y));
        acc_re[h] = __ffma2_rn(amp, cs, acc_re[h]);
        acc_im[h] = __ffma2_rn(amp, make_float2(sin_approx(ang.x), sin_approx(ang.y)), acc_im[h]);
    }
}

// Largest |t_z| max|dl| of a record the column step takes: (1 + j e) errs from e^{j e} by
// e^2 / 2 <= 2e-6 of the term.  On the 8 um and 3.74 um grids of 1920 and 3840 columns,
// max|dl| <= 0.0095 / m, so every record with |mu_z| <= 33 mm qualifies.
constexpr float kStepEps = 2e-3f;

// Pixel p of a thread's PX in the packed layout: pack and lane.  Layout 0 pairs neighbours
// (p = 2h, 2h + 1).  Layout 1 (the column-step configurations) pairs p = 4k + {0, 2} in pack 2k and
// p = 4k + {1, 3} in pack 2k + 1, so that each lane of an odd pack sits one column right of the
// same lane of the even pack before it.
template <int LAYOUT>
__host__ __device__ constexpr int pix_of(int h, int lane) {
    return LAYOUT == 0 ? 2 * h + lane : (h & 1) + 4 * (h >> 1) + 2 * lane;
}

// Column-step variant of splat_record (layout 1): the even packs as in splat_record; each odd
// pack, one column right, takes its linear forms a', b', g as the even pack's plus the record's
// per-column steps (x-slope dfx + z-slope sbar, the thread's mean step of f_z, plus the z-slope
// times the pixel's residual step dl: exact up to rounding) and its phase factor e^{j phi} as the even pack's
// times e^{j beta} (beta = t_x dfx + t_z sbar, one sin/cos per record and thread) times
// (1 + j t_z dl) for the residual.  The first-order residual errs by (t_z dl)^2 / 2: the cull
// sends a chunk to splat_record instead whenever a record's |t_z| max|dl| over the tile exceeds
// kStepEps.  The odd packs need no sin/cos of their own: per record and thread, 2 sin/cos in
// place of 8, for 8 more FP32 lane-ops per odd pack (36 against 28).
template <int PH>
__device__ __forceinline__ void splat_record_step(const float4 *__restrict__ sv, float dy, float dxm,
                                                  const float2 *ddx, const float2 *dz, const float2 *lfz,
                                                  const float2 *dl, float sbar, float2 *acc_re, float2 *acc_im) {
    const float4 Ar = sv[0], Br = sv[1], Gr = sv[2], Mr = sv[3], Xr = sv[4];
    const float2 ar = pair(fmaf(Ar.x, dxm, fmaf(Ar.y, dy, Ar.w))), br = pair(fmaf(Br.x, dxm, fmaf(Br.y, dy, Br.w)));
    const float2 gr = pair(fmaf(Gr.x, dxm, fmaf(Gr.y, dy, Gr.w)));
    const float t0 = fmaf(Mr.x, dxm, fmaf(Mr.y, dy, Mr.w));
    const float k0 = __fadd_rn(fmaf(t0, 0.15915494309189535f, 12582912.0f), -12582912.0f);
    const float2 tr = pair(fmaf(k0, -6.28318530717958647692f, t0));
    const float2 ax = pair(Ar.x), az = pair(Ar.z), bx = pair(Br.x), bz = pair(Br.z);
    const float2 gx = pair(Gr.x), gz = pair(Gr.z), tx2 = pair(Mr.x), tz = pair(Mr.z);
    // one column to the right: Xr = dfx (a'_x, b'_x, g_x, t_x); beta reduced to [-pi, pi]
    const float beta0 = fmaf(Mr.z, sbar, Xr.w);
    const float kb = __fadd_rn(fmaf(beta0, 0.15915494309189535f, 12582912.0f), -12582912.0f);
    const float beta = fmaf(kb, -6.28318530717958647692f, beta0);
    const float sb = sin_approx(beta);
    const float2 qc = pair(cos_approx(beta)), qs = pair(sb), nqs = pair(-sb);
    const float2 ca = pair(fmaf(Ar.z, sbar, Xr.x)), cb = pair(fmaf(Br.z, sbar, Xr.y));
    const float2 cg = pair(fmaf(Gr.z, sbar, Xr.z));
#pragma unroll
    for (int h = 0; h + 1 < PH; h += 2) {
        const float2 a = __ffma2_rn(az, dz[h], __ffma2_rn(ax, ddx[h], ar));
        const float2 b = __ffma2_rn(bz, dz[h], __ffma2_rn(bx, ddx[h], br));
        const float2 g = __ffma2_rn(gz, dz[h], __ffma2_rn(gx, ddx[h], gr));
        const float2 ang = __ffma2_rn(tz, dz[h], __ffma2_rn(tx2, ddx[h], tr));
        const float2 u = __ffma2_rn(a, a, __ffma2_rn(b, b, lfz[h]));
        const float2 amp = __fmul2_rn(g, make_float2(with_sign_of(ex2_approx(-u.x), g.x),
                                                     with_sign_of(ex2_approx(-u.y), g.y)));
        const float2 cs = make_float2(cos_approx(ang.x), cos_approx(ang.y));
        const float2 sn = make_float2(sin_approx(ang.x), sin_approx(ang.y));
        acc_re[h] = __ffma2_rn(amp, cs, acc_re[h]);
        acc_im[h] = __ffma2_rn(amp, sn, acc_im[h]);
        // the odd pack h + 1, one column right of pack h
        const float2 d = dl[h / 2];
        const float2 a1 = __ffma2_rn(az, d, __fadd2_rn(a, ca));
        const float2 b1 = __ffma2_rn(bz, d, __fadd2_rn(b, cb));
        const float2 g1 = __ffma2_rn(gz, d, __fadd2_rn(g, cg));
        const float2 u1 = __ffma2_rn(a1, a1, __ffma2_rn(b1, b1, lfz[h + 1]));
        const float2 amp1 = __fmul2_rn(g1, make_float2(with_sign_of(ex2_approx(-u1.x), g1.x),
                                                       with_sign_of(ex2_approx(-u1.y), g1.y)));
        const float2 e = __fmul2_rn(tz, d);              // residual phase step t_z dl
        const float2 pr = __ffma2_rn(e, nqs, qc);        // Re e^{j beta} (1 + j e)
        const float2 pi = __ffma2_rn(e, qc, qs);         // Im
        const float2 c1 = __ffma2_rn(neg2(sn), pi, __fmul2_rn(cs, pr));
        const float2 s1 = __ffma2_rn(sn, pr, __fmul2_rn(cs, pi));
        acc_re[h + 1] = __ffma2_rn(amp1, c1, acc_re[h + 1]);
        acc_im[h + 1] = __ffma2_rn(amp1, s1, acc_im[h + 1]);
    }
}

// RU: listed records evaluated per iteration (2: two independent accumulator sets for more
// instruction-level parallelism; needs the register room of the 4-pixel configuration)
// STEP: the column-step evaluation of the odd packs (splat_record_step, pixel layout 1).
template <int TW, int TH, int PX, int CHUNK, int STAGES, int RU, int MINB, int NPOLY, int STEP>
__global__ void __launch_bounds__((TW / PX) * TH, MINB) k_splat_mixed(const __grid_constant__ SplatArgs A) {
    constexpr int NT = (TW / PX) * TH;
    constexpr int SVN = STEP ? 5 : 4;  // float4 per record of the per-(record, tile) scalars
    constexpr int NW = NT / 32;          // warps = row bands of the tile
    constexpr int RPW = 32 / (TW / PX);  // tile rows per warp
    // records unrolled in the hot loop (four measured best; two where three CTAs share an SM's registers)
    constexpr int UNR = MINB >= 3 ? 2 : 4;
    // a chunk holds up to one record per thread (threads past the chunk cull nothing)
    static_assert(CHUNK <= NT && CHUNK <= 256 && CHUNK % 32 == 0 && (TW / PX) <= 32 && 32 % (TW / PX) == 0,
                  "chunk / tile shape");
    extern __shared__ __align__(128) unsigned char smem_raw[];
    Rec *s_rec = reinterpret_cast<Rec *>(smem_raw);
    float4 *s_sv = reinterpret_cast<float4 *>(smem_raw + sizeof(Rec) * STAGES * CHUNK);
    // per consumer warp w and source warp v: the chunk slots culled in by warp v that warp w
    // evaluates (records whose footprint meets w's band of rows)
    unsigned char *s_list =
        reinterpret_cast<unsigned char *>(smem_raw + sizeof(Rec) * STAGES * CHUNK + sizeof(float4) * SVN * CHUNK);
    __shared__ uint64_t s_full[STAGES];
    __shared__ uint64_t s_never;
    __shared__ unsigned char s_cnt[NW][NW];
    __shared__ float s_dzt;  // the current tile's bound on |f_z - 1/lambda|
    __shared__ unsigned s_dlmax;  // STEP: largest |dl| of the tile's threads (float bits, >= 0)
    __shared__ int s_item;

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (tid == 0) {
#pragma unroll
        for (int st = 0; st < STAGES; ++st) mbar_init(&s_full[st], 1);
        mbar_init(&s_never, 1);
        fence_mbar_init();
    }
    __syncthreads();
    uint32_t parity = 0;

    for (;;) {
        if (tid == 0) {
            s_item = atomicAdd(A.queue, 1);
            s_dlmax = 0u;
        }
        __syncthreads();
        const int it = s_item;
        if (it >= A.n_items) break;
        const unsigned item = A.items[it];
        const int seg = (int)(item / (unsigned)A.n_tiles), tile = (int)(item % (unsigned)A.n_tiles);
        if (!in_bounds(seg < A.segs.n_scenes * A.segs.n_lambda, A.status)) {  // checking build only
            __syncthreads();
            continue;
        }
        const int scene = seg / A.segs.n_lambda, l = seg % A.segs.n_lambda;
        int count = A.item_count[item];
        if (!in_bounds(count >= 0 && count <= seg_size(A.segs, seg), A.status)) count = 0;
        const Rec *rbase = A.rec + seg_start(A.segs, seg);
        const int tx = tile % A.tiles_x, ty = tile / A.tiles_x;
        const int c_lo = tx * TW, r_lo = ty * TH;
        const int c_hi = min(c_lo + TW, A.W) - 1, r_hi = min(r_lo + TH, A.H) - 1;
        const double inv_lam = A.inv_lam[l];
        const double k2 = inv_lam * inv_lam;
        // reference frequency f0 of the tile: the centre of its valid pixels, or -- if that is
        // evanescent -- its pixel nearest to f = 0, so that every |f - f0| stays within the tile
        int c_ref, r_ref;
        tile_ref(c_lo, c_hi, r_lo, r_hi, A.H, A.W, A.dfx, A.dfy, k2, c_ref, r_ref);
        const double f0x = (double)(c_ref - A.W / 2) * A.dfx, f0y = (double)(r_ref - A.H / 2) * A.dfy;
        const double f0z = sqrt(fmax(k2 - (f0x * f0x + f0y * f0y), 0.0));
        const float f0xf = (float)f0x, f0yf = (float)f0y, f0zf = (float)f0z, dz0f = (float)(f0z - inv_lam);

        // this thread's pixels: row prow, columns pcol0 .. pcol0 + PX - 1; (f_z - f0_z, log2(1/f_z))
        // from the per-call table built in FP64 for these tiles (k_pixtab)
        const int prow = r_lo + tid / (TW / PX);
        const int pcol0 = c_lo + (tid % (TW / PX)) * PX;
        const float dfxf = (float)A.dfx, dfyf = (float)A.dfy;
        const float dy = (float)((double)(prow - r_ref) * A.dfy);
        const float2 *prow_tab = A.pixtab + ((size_t)l * A.H + (prow < A.H ? prow : 0)) * A.W;
        // pixel pix_of(h, lane) is lane `lane` of the f32x2 pair h of the packed arithmetic
        constexpr int PH = PX / 2;
        float2 dx[PH], dz[PH], lfz[PH];  // dx: offsets from the thread's middle column
        const float dxm = (float)(pcol0 + PX / 2 - c_ref) * dfxf;
#pragma unroll
        for (int h = 0; h < PH; ++h) {
#pragma unroll
            for (int ln = 0; ln < 2; ++ln) {
                const int p = pix_of<STEP>(h, ln);
                const int col = pcol0 + p;
                const float2 pt = (prow < A.H && col < A.W) ? prow_tab[col] : make_float2(0.f, -INFINITY);
                const bool ok = pt.y > -INFINITY;  // (0, -inf): evanescent or outside the grid
                const float vx = (float)(p - PX / 2) * dfxf;
                const float vl = ok ? -pt.y : INFINITY;  // log2 f_z: 2^-(a^2 + b^2 + log2 f_z) = f_z^-1 2^-(a^2 + b^2)
                const float vz = ok ? pt.x : 0.f;
                if (ln) {
                    dx[h].y = vx;
                    lfz[h].y = vl;
                    dz[h].y = vz;
                } else {
                    dx[h].x = vx;
                    lfz[h].x = vl;
                    dz[h].x = vz;
                }
            }
        }
        // STEP: the thread's mean step of f_z from an even pack's pixel to the odd pack's one
        // column right (sbar), each pixel's residual from it (dl), and the tile's largest |dl|.
        // A pixel without amplitude (lfz = inf) needs no phase; an even one whose right
        // neighbour has amplitude takes f_z - f0_z = the neighbour's minus sbar, so that its
        // residual is 0 (only its phase is carried to the neighbour).
        float sbar = 0.f;
        float2 dl[PH / 2 > 0 ? PH / 2 : 1];
        if constexpr (STEP) {
            float ssum = 0.f;
            int ns = 0;
#pragma unroll
            for (int h = 0; h + 1 < PH; h += 2) {
                if (lfz[h].x < INFINITY && lfz[h + 1].x < INFINITY) {
                    ssum += dz[h + 1].x - dz[h].x;
                    ++ns;
                }
                if (lfz[h].y < INFINITY && lfz[h + 1].y < INFINITY) {
                    ssum += dz[h + 1].y - dz[h].y;
                    ++ns;
                }
            }
            sbar = ns ? ssum / (float)ns : 0.f;
            float dmax = 0.f;
#pragma unroll
            for (int h = 0; h + 1 < PH; h += 2) {
                float d0 = 0.f, d1 = 0.f;
                if (lfz[h + 1].x < INFINITY) {
                    if (lfz[h].x < INFINITY) d0 = (dz[h + 1].x - dz[h].x) - sbar;
                    else dz[h].x = dz[h + 1].x - sbar;
                }
                if (lfz[h + 1].y < INFINITY) {
                    if (lfz[h].y < INFINITY) d1 = (dz[h + 1].y - dz[h].y) - sbar;
                    else dz[h].y = dz[h + 1].y - sbar;
                }
                dl[h / 2] = make_float2(d0, d1);
                dmax = fmaxf(dmax, fmaxf(fabsf(d0), fabsf(d1)));
            }
            const unsigned m = __reduce_max_sync(0xffffffffu, __float_as_uint(dmax));
            if (lane == 0) atomicMax(&s_dlmax, m);  // read by the cull, after the barrier that opens each chunk
        }
        // tile rectangle (pixel-centre frequencies of the valid pixels) for the cull
        const float x0 = (float)((double)(c_lo - A.W / 2) * A.dfx), x1 = (float)((double)(c_hi - A.W / 2) * A.dfx);
        const float y0 = (float)((double)(r_lo - A.H / 2) * A.dfy), y1 = (float)((double)(r_hi - A.H / 2) * A.dfy);
        if (tid == 0)  // read by the cull, after the barrier that opens each chunk
            s_dzt = (float)dz_far((double)(c_lo - A.W / 2) * A.dfx, (double)(c_hi - A.W / 2) * A.dfx,
                                  (double)(r_lo - A.H / 2) * A.dfy, (double)(r_hi - A.H / 2) * A.dfy, inv_lam);

        const int n_chunks = (count + CHUNK - 1) / CHUNK;
        int issued = 0, consumed = 0;
        if (tid == 0) fence_proxy_async();
        for (; issued < min(STAGES, n_chunks); ++issued) {
            if (tid == 0) {
                const int st = issued % STAGES;
                const int nrec = min(CHUNK, count - issued * CHUNK);
                mbar_expect_tx(&s_full[st], (uint32_t)(nrec * sizeof(Rec)));
                bulk_g2s(s_rec + st * CHUNK, rbase + (long long)issued * CHUNK, (uint32_t)(nrec * sizeof(Rec)),
                         &s_full[st]);
            }
        }

        float2 acc_re[PH], acc_im[PH], acc2_re[PH], acc2_im[PH];
        float sum_re[PX], sum_im[PX], cmp_re[PX], cmp_im[PX];
#pragma unroll
        for (int h = 0; h < PH; ++h) acc_re[h] = acc_im[h] = acc2_re[h] = acc2_im[h] = make_float2(0.f, 0.f);
#pragma unroll
        for (int p = 0; p < PX; ++p) sum_re[p] = sum_im[p] = cmp_re[p] = cmp_im[p] = 0.f;

        bool timed_out = false;
        if (A.debug & GWS_DEBUG_FORCE_TIMEOUT) {
            // a barrier nothing arrives on: exercises the bounded wait and the drain
            bool ok = mbar_wait_bounded(&s_never, 0, A.timeout);
            timed_out = __syncthreads_or(!ok) != 0;
        }
        for (int ch = 0; ch < n_chunks && !timed_out; ++ch) {
            const int st = ch % STAGES;
            const bool ok = mbar_wait_bounded(&s_full[st], (parity >> st) & 1u, A.timeout);
            if (__syncthreads_or(!ok)) {
                timed_out = true;
                break;
            }
            parity ^= (1u << st);
            consumed = ch + 1;

            // ---- cull + per-(record, tile) scalars (one thread per record) ----
            // A record survives if its footprint ellipse meets the tile; it is then tested
            // against each warp's band of RPW rows (FP32, from the tile's edges), and only the
            // warps whose band it meets evaluate it.
            const int nrec = min(CHUNK, count - ch * CHUNK);
            bool need_direct = false;  // STEP: this record's residual phase step is too large for it
            {
                unsigned bands = 0;
                if (tid < nrec) {
                    const Rec &r = s_rec[st * CHUNK + tid];
                    // the footprint for this tile's bound on |d_z| (within the grid-wide one)
                    const float sc = footprint_scale(A.dzmax[l], s_dzt, r.wz);
                    const float e00 = r.e00 * sc, e01 = r.e01 * sc, e11 = r.e11 * sc;
                    if (ellipse_hits_rect(e00, e01, e11, x0, x1, y0, y1)) {
#pragma unroll
                        for (int w = 0; w < NW; ++w) {
                            const float yb0 = fmaf((float)(w * RPW), dfyf, y0);
                            const float yb1 = fminf(fmaf((float)(RPW - 1), dfyf, yb0), y1);
                            if (yb0 <= y1 && ellipse_hits_rect(e00, e01, e11, x0, x1, yb0, yb1)) bands |= 1u << w;
                        }
                    }
                    if (bands) {
                        double cyc = -(f0x * r.mux + f0y * r.muy + f0z * r.muz);
                        if (A.phase_match) cyc += r.muz * inv_lam;
                        cyc -= rint(cyc);
                        cyc *= kTwoPi;  // radians
                        const float a0 = fmaf(r.r1z, dz0f, fmaf(r.r1y, f0yf, r.r1x * f0xf));
                        const float b0 = fmaf(r.r2z, dz0f, fmaf(r.r2y, f0yf, r.r2x * f0xf));
                        const float g0 = fmaf(r.r3z, f0zf, fmaf(r.r3y, f0yf, r.r3x * f0xf));
                        float4 *sv = s_sv + tid * SVN;
                        sv[0] = make_float4(r.r1x, r.r1y, r.r1z, a0);
                        sv[1] = make_float4(r.r2x, r.r2y, r.r2z, b0);
                        sv[2] = make_float4(r.r3x, r.r3y, r.r3z, g0);
                        sv[3] = make_float4(r.mx, r.my, r.mz, (float)cyc);
                        if constexpr (STEP) {
                            sv[4] = make_float4(r.r1x * dfxf, r.r2x * dfxf, r.r3x * dfxf, r.mx * dfxf);
                            need_direct = fabsf(r.mz) * __uint_as_float(s_dlmax) > kStepEps;
                        }
                    }
                }
                const unsigned lt = (1u << lane) - 1u;
#pragma unroll
                for (int w = 0; w < NW; ++w) {
                    const bool mine = (bands >> w) & 1u;
                    const unsigned bal = __ballot_sync(0xffffffffu, mine);
                    if (mine) s_list[(w * NW + warp) * 32 + __popc(bal & lt)] = (unsigned char)(tid & 255);
                    if (lane == 0) s_cnt[w][warp] = (unsigned char)__popc(bal);
                }
            }
            // STEP: the whole chunk goes through splat_record if any of its records needs it
            bool direct = true;
            if constexpr (STEP) direct = __syncthreads_or(need_direct) != 0;
            else __syncthreads();
            // the stage is free again: refill it with the chunk STAGES ahead
            if (issued < n_chunks) {
                if (tid == 0) {
                    fence_proxy_async();
                    const int sti = issued % STAGES;
                    const int nr = min(CHUNK, count - issued * CHUNK);
                    mbar_expect_tx(&s_full[sti], (uint32_t)(nr * sizeof(Rec)));
                    bulk_g2s(s_rec + sti * CHUNK, rbase + (long long)issued * CHUNK, (uint32_t)(nr * sizeof(Rec)),
                             &s_full[sti]);
                }
                ++issued;
            }

            // ---- the hot loop: every surviving record x this thread's PX pixels ----
            for (int v = 0; v < NW; ++v) {
                int cnt = s_cnt[warp][v];
                const unsigned char *lst = s_list + (warp * NW + v) * 32;
#ifdef GWS_CHECK_BOUNDS
                // every listed slot must hold a record of this chunk
                for (int i = 0; i < cnt; ++i)
                    if (!in_bounds(lst[i] < nrec, A.status)) cnt = 0;
#endif
                int i = 0;
                if constexpr (STEP) {
                    if (!direct) {
#pragma unroll(UNR)
                        for (; i < cnt; ++i)
                            splat_record_step<PH>(s_sv + lst[i] * SVN, dy, dxm, dx, dz, lfz, dl, sbar, acc_re, acc_im);
                        continue;
                    }
                }
                if (RU == 2) {
                    for (; i + 1 < cnt; i += 2) {
                        splat_record<PH, NPOLY>(s_sv + lst[i] * SVN, dy, dxm, dx, dz, lfz, acc_re, acc_im);
                        splat_record<PH, NPOLY>(s_sv + lst[i + 1] * SVN, dy, dxm, dx, dz, lfz, acc2_re, acc2_im);
                    }
                }
#pragma unroll(UNR)
                for (; i < cnt; ++i)
                    splat_record<PH, NPOLY>(s_sv + lst[i] * SVN, dy, dxm, dx, dz, lfz, acc_re, acc_im);
            }
            if (RU == 2) {
#pragma unroll
                for (int h = 0; h < PH; ++h) {
                    acc_re[h] = __fadd2_rn(acc_re[h], acc2_re[h]);
                    acc_im[h] = __fadd2_rn(acc_im[h], acc2_im[h]);
                    acc2_re[h] = acc2_im[h] = make_float2(0.f, 0.f);
                }
            }
#pragma unroll
            for (int h = 0; h < PH; ++h) {
                const int p0 = pix_of<STEP>(h, 0), p1 = pix_of<STEP>(h, 1);
                two_sum_acc(sum_re[p0], cmp_re[p0], acc_re[h].x);
                two_sum_acc(sum_re[p1], cmp_re[p1], acc_re[h].y);
                two_sum_acc(sum_im[p0], cmp_im[p0], acc_im[h].x);
                two_sum_acc(sum_im[p1], cmp_im[p1], acc_im[h].y);
                acc_re[h] = acc_im[h] = make_float2(0.f, 0.f);
            }
            __syncthreads();
        }

        if (timed_out) {
            if (tid == 0) atomicOr(A.status, ST_TIMEOUT);
            // wait (bounded) for this CTA's own copies still in flight, then leave
            for (int ch = consumed; ch < issued; ++ch) {
                const int st = ch % STAGES;
                mbar_wait_bounded(&s_full[st], (parity >> st) & 1u, 4ull * A.timeout + 100000ull);
                parity ^= (1u << st);
            }
            return;
        }

        // ---- epilogue: compensated total, centred-DFT pre-modulation, store ----
        if (prow < A.H) {
            float2 *out = reinterpret_cast<float2 *>(A.out[scene]) + (size_t)l * A.H * A.W + (size_t)prow * A.W;
            const long long hw = (long long)A.H * A.W;
            const float inv_hw = 1.0f / (float)hw;
#pragma unroll
            for (int p = 0; p < PX; ++p) {
                const int col = pcol0 + p;
                if (col < A.W) {
                    float re = sum_re[p] + cmp_re[p], im = sum_im[p] + cmp_im[p];
                    if (A.field_mode) {  // e^{-j2pi(m r0/H + n c0/W)}, the angle an exact integer over H W
                        if (((A.H | A.W) & 1) == 0) {  // even grid: (-1)^(r + c) exactly
                            if ((prow + col) & 1) {
                                re = -re;
                                im = -im;
                            }
                        } else {
                            long long num = mod_num2(prow, A.H / 2, 1, col, A.W / 2, 1, A.H, A.W);
                            if (2 * num > hw) num -= hw;
                            float sn, cs;
                            sincospif(-2.0f * (float)num * inv_hw, &sn, &cs);
                            const float r2 = re * cs - im * sn;
                            im = re * sn + im * cs;
                            re = r2;
                        }
                    }
                    out[col] = make_float2(re, im);
                }
            }
        }
        __syncthreads();
    }
}

// ---- tile configurations (autotuned) ----------------------------------------------------

// MINB: CTAs per SM the launch bounds aim at (3 needs <= 85 registers and the 2-stage ring);
// CHUNK: Gaussian records per bulk-copied chunk (<= threads; 0 = one per thread); STAGES: ring depth
template <int TW, int TH, int PX, int RU = 1, int STAGES = 3, int MINB = 2, int CHUNK_ = 0, int NPOLY = 0, int STEP = 0>
struct SplatCfg {
    static constexpr int NT = (TW / PX) * TH;
    static constexpr int CHUNK = CHUNK_ > 0 ? CHUNK_ : NT;
    static constexpr size_t smem =
        sizeof(Rec) * STAGES * CHUNK + sizeof(float4) * (STEP ? 5 : 4) * CHUNK + (size_t)(NT / 32) * NT;
    // the opt-in shared-memory size is a per-device function attribute: set it once per
    // device (gws_prepare or the first call), not while a stream is being captured
    static cudaError_t prepare() {
        static bool done[64] = {false};
        int dev = 0;
        cudaError_t e = cudaGetDevice(&dev);
        if (e != cudaSuccess) return e;
        if (dev >= 0 && dev < 64 && done[dev]) return cudaSuccess;
        e = cudaFuncSetAttribute(k_splat_mixed<TW, TH, PX, CHUNK, STAGES, RU, MINB, NPOLY, STEP>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e == cudaSuccess && dev >= 0 && dev < 64) done[dev] = true;
        return e;
    }
    static cudaError_t launch(const SplatArgs &a, int grid, cudaStream_t s) {
        cudaError_t e = prepare();
        if (e != cudaSuccess) return e;
        k_splat_mixed<TW, TH, PX, CHUNK, STAGES, RU, MINB, NPOLY, STEP><<<grid, NT, smem, s>>>(a);
        count_launches(1);
        return cudaGetLastError();
    }
};

// The autotuner's search space: tile shape (frequencies per CTA), pixels per thread, records per
// iteration, Gaussian records per chunk, ring depth and CTAs per SM.
using Cfg1 = SplatCfg<64, 32, 8>;                 // 64x32, 8 px/thread, 256 records/chunk, 3 stages
using Cfg2 = SplatCfg<32, 32, 4>;                 // 32x32, 4 px/thread
using Cfg3 = SplatCfg<128, 16, 8>;                // 128x16
using Cfg4 = SplatCfg<32, 32, 4, 2>;              // 32x32, two records per iteration
using Cfg5 = SplatCfg<32, 32, 4, 1, 2, 3>;        // 32x32 at three CTAs per SM, 2 stages
using Cfg6 = SplatCfg<64, 32, 8, 1, 4, 2, 128>;   // 64x32, 128 records/chunk, 4 stages
using Cfg7 = SplatCfg<64, 32, 8, 1, 2, 2, 256>;   // 64x32, 256 records/chunk, 2 stages
using Cfg8 = SplatCfg<64, 32, 8, 1, 6, 2, 64>;    // 64x32, 64 records/chunk, 6 stages
using Cfg9 = SplatCfg<64, 32, 8, 1, 3, 2, 0, 1>;  // 64x32, the cos of 1 of the 4 pixel pairs on the FP32 pipe
using Cfg10 = SplatCfg<128, 16, 8, 1, 3, 2, 0, 1>;  // 128x16, likewise
using Cfg11 = SplatCfg<64, 32, 8, 1, 3, 2, 0, 0, 1>;  // 64x32, the odd packs by the column step
using Cfg12 = SplatCfg<128, 16, 8, 1, 3, 2, 0, 0, 1>; // 128x16, likewise

cudaError_t prepare_splat_kernels() {
    cudaError_t e = Cfg1::prepare();
    if (e == cudaSuccess) e = Cfg2::prepare();
    if (e == cudaSuccess) e = Cfg3::prepare();
    if (e == cudaSuccess) e = Cfg4::prepare();
    if (e == cudaSuccess) e = Cfg5::prepare();
    if (e == cudaSuccess) e = Cfg6::prepare();
    if (e == cudaSuccess) e = Cfg7::prepare();
    if (e == cudaSuccess) e = Cfg8::prepare();
    if (e == cudaSuccess) e = Cfg9::prepare();
    if (e == cudaSuccess) e = Cfg10::prepare();
    if (e == cudaSuccess) e = Cfg11::prepare();
    if (e == cudaSuccess) e = Cfg12::prepare();
    return e;
}

template <typename C>
constexpr TileCfg describe(int id, int tw, int th, int px, int ru, int stages, int ctas, int npoly = 0, int step = 0) {
    return TileCfg{id, tw, th, px, ru, C::CHUNK, stages, ctas, npoly, step};
}
static const TileCfg kCfgs[] = {
    describe<Cfg1>(1, 64, 32, 8, 1, 3, 2), describe<Cfg2>(2, 32, 32, 4, 1, 3, 2), describe<Cfg3>(3, 128, 16, 8, 1, 3, 2),
    describe<Cfg4>(4, 32, 32, 4, 2, 3, 2), describe<Cfg5>(5, 32, 32, 4, 1, 2, 3), describe<Cfg6>(6, 64, 32, 8, 1, 4, 2),
    describe<Cfg7>(7, 64, 32, 8, 1, 2, 2), describe<Cfg8>(8, 64, 32, 8, 1, 6, 2), describe<Cfg9>(9, 64, 32, 8, 1, 3, 2, 1),
    describe<Cfg10>(10, 128, 16, 8, 1, 3, 2, 1), describe<Cfg11>(11, 64, 32, 8, 1, 3, 2, 0, 1),
    describe<Cfg12>(12, 128, 16, 8, 1, 3, 2, 0, 1)};

int n_tile_cfgs() { return (int)(sizeof(kCfgs) / sizeof(kCfgs[0])); }
TileCfg tile_cfg(int id) {
    if (id < 1 || id > n_tile_cfgs()) id = 1;
    return kCfgs[id - 1];
}
int splat_mixed_ctas_per_sm(int cfg) { return tile_cfg(cfg).ctas; }

cudaError_t launch_splat_mixed(int cfg, const SplatArgs &a, int grid, cudaStream_t s) {
    switch (cfg) {
        case 2: return Cfg2::launch(a, grid, s);
        case 3: return Cfg3::launch(a, grid, s);
        case 4: return Cfg4::launch(a, grid, s);
        case 5: return Cfg5::launch(a, grid, s);
        case 6: return Cfg6::launch(a, grid, s);
        case 7: return Cfg7::launch(a, grid, s);
        case 8: return Cfg8::launch(a, grid, s);
        case 9: return Cfg9::launch(a, grid, s);
        case 10: return Cfg10::launch(a, grid, s);
        case 11: return Cfg11::launch(a, grid, s);
        case 12: return Cfg12::launch(a, grid, s);
        default: return Cfg1::launch(a, grid, s);
    }
}

// ---- plain FP64 path: one thread per frequency pixel, every Gaussian, no truncation ----

__global__ void __launch_bounds__(256) k_splat_fp64(const __grid_constant__ Splat64Args A) {
    const int c = blockIdx.x * 16 + threadIdx.x;
    const int r = blockIdx.y * 16 + threadIdx.y;
    const int seg = blockIdx.z;
    const int scene = seg / A.segs.n_lambda, l = seg % A.segs.n_lambda;
    if (r >= A.H || c >= A.W) return;
    const double inv_lam = A.inv_lam[l];
    const double fx = (double)(c - A.W / 2) * A.dfx, fy = (double)(r - A.H / 2) * A.dfy;
    const double rho2 = fx * fx + fy * fy, k2 = inv_lam * inv_lam;
    double sre = 0.0, sim = 0.0;
    if (rho2 < k2) {
        const double fz = sqrt(k2 - rho2);
        const double dz = fz - inv_lam;
        const long long p0 = A.segs.off[scene], p1 = A.segs.off[scene + 1];
        const int L = A.segs.n_lambda;
        if (!in_bounds(scene < A.segs.n_scenes && p0 >= 0 && p1 >= p0, A.status)) return;
        for (long long p = p0; p < p1; ++p) {
            const Rec64 &g = A.rec[p];
            const double w = A.w[p * L + l];
            const double a = g.r1[0] * fx + g.r1[1] * fy + g.r1[2] * dz;
            const double b = g.r2[0] * fx + g.r2[1] * fy + g.r2[2] * dz;
            const double gg = g.r3[0] * fx + g.r3[1] * fy + g.r3[2] * fz;
            const double amp = w * kTwoPi * g.su * g.sv * fabs(gg) / fz *
                               exp(-2.0 * kPi * kPi * (g.su * g.su * a * a + g.sv * g.sv * b * b));
            double cyc = -(fx * g.mu[0] + fy * g.mu[1] + fz * g.mu[2]);
            if (A.phase_match) cyc += g.mu[2] * inv_lam;
            cyc -= rint(cyc);
            double sn, cs;
            sincospi(2.0 * cyc, &sn, &cs);
            sre += amp * cs;
            sim += amp * sn;
        }
    }
    if (A.field_mode) {
        const long long hw = (long long)A.H * A.W;
        long long num = mod_num2(r, A.H / 2, 1, c, A.W / 2, 1, A.H, A.W);
        if (2 * num > hw) num -= hw;
        double sn, cs;
        sincospi(-2.0 * (double)num / (double)hw, &sn, &cs);
        const double t = sre * cs - sim * sn;
        sim = sre * sn + sim * cs;
        sre = t;
    }
    double2 *out = reinterpret_cast<double2 *>(A.out[scene]) + (size_t)l * A.H * A.W + (size_t)r * A.W + c;
    *out = make_double2(sre, sim);
}

cudaError_t launch_splat_fp64(const Splat64Args &a, cudaStream_t s) {
    dim3 grid((a.W + 15) / 16, (a.H + 15) / 16, a.segs.n_scenes * a.segs.n_lambda);
    k_splat_fp64<<<grid, dim3(16, 16), 0, s>>>(a);
    count_launches(1);
    return cudaGetLastError();
}

}  // namespace gws
