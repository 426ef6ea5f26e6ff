/*
 * gws.h -- C ABI of libgws, the GB300 (sm_103a) hot path of Gaussian Wave Splatting
 * (Choi et al., "Gaussian Wave Splatting for Computer-Generated Holography", arXiv
 * 2505.06582).
 *
 * What the library computes (paper sections / equations in brackets):
 *   N 2D Gaussians in hologram space -> the complex field at the SLM plane.
 *   - Each Gaussian i has a mean mu_i (3D), a rotation q_i (unit quaternion, columns
 *     r1 = t_u, r2 = t_v, r3 = normal) and scales s_u, s_v [Sec. 3], an opacity o_i
 *     [Eq. 2] and a per-wavelength amplitude c_il [Eq. 5].
 *   - Its angular spectrum at the SLM is the closed form of Eq. 10 evaluated on the
 *     tilted-plane remapped frequencies with the Jacobian det J = k_oz / k_z and the
 *     reference-wave shift f_r = (0, 0, 1/lambda) [Sec. 4.1, Eq. 9-10, supplement Sec. 1.2]:
 *        u_i(f) = 2 pi s_u s_v |r3.f| / f_z exp(-2 pi^2 [s_u^2 (r1.d)^2 + s_v^2 (r2.d)^2])
 *                 exp(-j 2 pi f.mu_i),     d = f - f_r,  f_z = sqrt(1/lambda^2 - fx^2 - fy^2)
 *     in ordinary frequency (cycles/m); zero outside fx^2 + fy^2 < 1/lambda^2 [Eq. 4].
 *   - Blending: the order-invariant Fourier-domain sum of Eq. 12,
 *        u_SLM(f) = sum_i c_il o_i u_i(f)                                (GWS_BLEND_OIT)
 *     or the depth-sorted transmittance variant of Eq. 5-6 with T_i held at the
 *     Gaussian's centre, T_i = prod_{j in front} (1 - alpha_j(mu_i)), alpha from Eq. 2 and
 *     the t_eps = 1/255 threshold of Algorithm S2                         (GWS_BLEND_SORTED_T).
 *   - One inverse FFT [Algorithm S1, S4; Eq. 3]: the field is the centred inverse DFT of
 *     u_SLM scaled by dfx dfy.
 *   - Double-phase encoding for a phase-only SLM [Sec. 5 and the supplement's phase
 *     encoding paragraph].
 *
 * Layouts (all row-major; row r <-> y, column c <-> x; centred grids):
 *   fx(c) = (c - floor(W/2)) / (W pitch_x),  fy(r) = (r - floor(H/2)) / (H pitch_y);
 *   field pixel (r, c) sits at x = (c - floor(W/2)) pitch_x, y = (r - floor(H/2)) pitch_y.
 *   Gaussians are structure-of-arrays: mean double[n][3] (m), quat float[n][4] (w,x,y,z,
 *   normalised inside), scale float[n][2] (m), opacity float[n], amp float[n][n_lambda].
 *   Fields / spectra are interleaved complex [n_lambda][H][W]: complex64 for
 *   GWS_PREC_MIXED, complex128 for GWS_PREC_FP64.
 *
 * Ownership: every array argument is caller-owned DEVICE memory except
 *   gws_slm.wavelengths (host, read during the call).  The call path never allocates:
 *   scratch lives in the caller's workspace (gws_opts.workspace, at least
 *   gws_workspace_size() bytes, 256-byte aligned).  The one exception is the cuFFT plan of
 *   a new grid shape, created (and allocated by cuFFT) by gws_prepare() or on the first
 *   call with that shape; call gws_prepare() before capturing calls into a CUDA graph.
 *
 * Errors: host-checkable argument errors return a gws_status synchronously and launch
 *   nothing.  Conditions only the device can see (non-finite inputs, opacity outside
 *   [0,1], non-positive scales, a zero quaternion, a wait that timed out) are recorded in
 *   a status word inside the workspace; read it with gws_get_device_status().  Calls are
 *   asynchronous on gws_opts.stream.  No exception crosses the ABI.  There is no CPU
 *   fallback: without a CUDA device every compute entry point returns GWS_ERR_CUDA.
 */
#ifndef GWS_H
#define GWS_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define GWS_API __attribute__((visibility("default")))
#else
#define GWS_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

#define GWS_ABI_VERSION 1
#define GWS_MAX_LAMBDA 16  /* wavelengths per call */
#define GWS_MAX_SCENES 128 /* scenes per batched call */

typedef enum {
    GWS_OK = 0,
    GWS_ERR_INVALID_ARG = 1, /* bad argument (host) or bad Gaussian value (device status) */
    GWS_ERR_WORKSPACE = 2,   /* workspace missing, too small or misaligned */
    GWS_ERR_CUDA = 3,        /* a CUDA / cuFFT call failed, or no device */
    GWS_ERR_NONFINITE = 4,   /* device status: NaN / Inf among the inputs */
    GWS_ERR_TIMEOUT = 5,     /* device status: a bounded wait gave up */
    GWS_ERR_UNSUPPORTED = 6, /* combination not implemented (e.g. FP64 backward) */
    GWS_ERR_BOUNDS = 7       /* device status, bounds-checking build only: an index out of range
                                (the access was skipped) or a workspace canary overwritten */
} gws_status;

typedef enum {
    GWS_BLEND_OIT = 0,      /* Eq. 12: order-invariant sum, T_i = 1 */
    GWS_BLEND_SORTED_T = 1, /* Eq. 5-6 with T_i at the Gaussian's centre (depth-sorted) */
    GWS_BLEND_EXACT = 2,    /* Eq. 5-6 with the spatial transmittance map (Algorithm S2): front to back,
                               u_SLM += c o F(T u_k) H(f, -z_k), T *= 1 - alpha_k, alpha_k = o |u_k|
                               above t_eps (or binarised at t_binarize); MIXED forward only */
    GWS_BLEND_PARTIAL_COHERENT = 3 /* Eq. 14 summed as Eq. 12: one time-multiplexed frame of partially
                               coherent GWS.  Each Gaussian's spectrum (Eq. 10 at the origin) is
                               convolved with the angular kernel K(f) = Y_l^m(k_hat) e^{j phi(f)}
                               (opts.pc_l, opts.pc_m; k_hat = lambda (f_x, f_y, f_z), K = 0 where
                               evanescent) and then translated by e^{-j 2 pi f . mu}: through the
                               spatial domain, its field on its own plane times
                               kappa(x) = sum_f K(f) e^{j 2 pi f . x} / sqrt(sum_f Y^2) (E|kappa|^2 = 1).
                               phi(f) = 2 pi u - pi, u = SplitMix64 output number
                               ((pc_frame L + l) H + r) W + c + 1 of the stream seeded with pc_seed
                               (top 53 bits / 2^53).  MIXED forward only, single scene */
} gws_blend;

typedef enum {
    GWS_PREC_FP64 = 0, /* every step in FP64, one thread per frequency pixel, no truncation */
    GWS_PREC_MIXED = 1 /* FP32 bulk, FP64 phase anchors, compensated sums, footprint truncation */
} gws_precision;

typedef enum {
    GWS_DOMAIN_FIELD = 0,   /* forward writes the SLM field (after the inverse FFT) */
    GWS_DOMAIN_SPECTRUM = 1 /* forward writes u_SLM(f) itself (no FFT); backward takes dL/du_SLM */
} gws_domain;

enum {
    GWS_DEBUG_FORCE_TIMEOUT = 1u, /* the splat kernel's first wait targets a barrier nothing
                                     arrives on: it gives up after timeout_cycles, records
                                     GWS_ERR_TIMEOUT and returns (tests the bounded waits) */
    GWS_DEBUG_TIME_KERNELS = 2u   /* record CUDA events around the splat / FFT / encode launches
                                     on opts.stream; read them with gws_kernel_time_ms() */
};

typedef enum { /* timers of GWS_DEBUG_TIME_KERNELS */
    GWS_TIMER_SPLAT_FWD = 0,
    GWS_TIMER_SPLAT_BWD = 1,
    GWS_TIMER_FFT = 2,
    GWS_TIMER_ENCODE = 3,
    GWS_TIMER_TOTAL = 4 /* the whole entry point */
} gws_timer;

typedef struct {
    const double *mean;   /* [n][3], metres */
    const float *quat;    /* [n][4], (w, x, y, z), any non-zero norm */
    const float *scale;   /* [n][2], (s_u, s_v) > 0, metres */
    const float *opacity; /* [n], in [0, 1] */
    const float *amp;     /* [n][n_lambda] */
} gws_gaussians;

typedef struct { /* gradients, same layout as gws_gaussians, device memory */
    double *mean;
    float *quat;
    float *scale;
    float *opacity;
    float *amp;
} gws_gaussians_grad;

typedef struct {
    int H, W;                  /* rows (y), columns (x) */
    double pitch_x, pitch_y;   /* metres */
    int n_lambda;              /* 1 .. GWS_MAX_LAMBDA */
    const double *wavelengths; /* HOST array [n_lambda], metres */
} gws_slm;

typedef struct {
    int blend;        /* gws_blend */
    int prec;         /* gws_precision */
    int domain;       /* gws_domain */
    int phase_match;  /* 1: multiply each Gaussian by exp(+j 2 pi mu_z / lambda) (supplement,
                         "we match the phase of each wavefront"); default 0 */
    float trunc_eps;  /* MIXED: relative amplitude below which a Gaussian's spectrum is cut
                         (footprint ellipse exp(-E) >= eps); default 1e-5 */
    float alpha_min;  /* SORTED_T: t_eps of Algorithm S2; default 1/255 */
    int tile_cfg;     /* MIXED: splat tile configuration, 0 = tuned / default */
    uint32_t debug_flags;    /* GWS_DEBUG_* */
    uint64_t timeout_cycles; /* bound of every device-side wait, in SM clock cycles */
    void *stream;            /* cudaStream_t (NULL = legacy default stream) */
    void *workspace;         /* device scratch, >= gws_workspace_size() bytes */
    size_t workspace_bytes;
    float t_binarize;        /* EXACT: > 0 binarises alpha (disk occlusion, Algorithm S2); default 0 */
    int exact_batch;         /* EXACT, PARTIAL_COHERENT: Gaussians per batch of fields in flight (0 = 128) */
    int pc_l, pc_m;          /* PARTIAL_COHERENT: degree 0..3 and order -l..l of the kernel's SH; default 0, 0 */
    uint64_t pc_seed;        /* PARTIAL_COHERENT: seed of the random phases; default 0 */
    uint64_t pc_frame;       /* PARTIAL_COHERENT: frame index t (independent phases per frame); default 0 */
    int pc_frames;           /* PARTIAL_COHERENT: frames pc_frame .. pc_frame + pc_frames - 1 in one call
                                (0 or 1: one frame; at most GWS_MAX_PC_FRAMES).  field_out then holds
                                pc_frames x n_lambda x H x W values, frame-major; each batch's fields on
                                their own planes are computed once and shared by the frames (the
                                workspace holds one more batch of fields and a kernel pattern per frame).
                                Every frame equals the single-frame call with that pc_frame. */
} gws_opts;

#define GWS_MAX_PC_FRAMES 64

/* Fills *o with the defaults listed above (OIT, MIXED, FIELD). */
GWS_API void gws_opts_default(gws_opts *o);

/* Human-readable name of a status code (static storage). */
GWS_API const char *gws_status_string(gws_status s);

/* Library version (GWS_ABI_VERSION). */
GWS_API int gws_version(void);

/* Workspace bytes needed by forward / backward / encode for scenes of sizes n[0..n_scenes)
 * on this SLM with these options (blend, prec, domain, tile_cfg matter).  Host only. */
GWS_API gws_status gws_workspace_size(const int64_t *n, int n_scenes, const gws_slm *slm, const gws_opts *opts,
                              size_t *bytes);

/* Per-device set-up for this grid on the current device: creates the cuFFT plans (batch
 * n_lambda; n_scenes * n_lambda for batched calls whose outputs are contiguous; the exact
 * blending batch; complex64 and, for FP64, complex128) and sets the kernels' shared-memory
 * attributes.  May allocate (inside cuFFT).  Call it before capturing gws_* calls into a
 * CUDA graph. */
GWS_API gws_status gws_prepare(const gws_slm *slm, const gws_opts *opts, int n_scenes);

/* Forward [Eq. 10, Eq. 12 or Eq. 5-6, Eq. 3]: field_out = centred inverse DFT of u_SLM
 * (domain FIELD) or u_SLM itself (domain SPECTRUM); complex [n_lambda][H][W], complex64
 * (MIXED) or complex128 (FP64).  n = 0 gives a zero field. */
GWS_API gws_status gws_forward(const gws_gaussians *g, int64_t n, const gws_slm *slm, const gws_opts *opts,
                       void *field_out);

/* Batched forward: n_scenes scenes (each its own arrays and size n[k]) on one SLM, one
 * persistent splat launch over every (scene, wavelength, frequency tile).  field_out[k]
 * as in gws_forward.  Results equal per-scene gws_forward calls bit for bit. */
GWS_API gws_status gws_forward_batched(const gws_gaussians *scenes, const int64_t *n, int n_scenes,
                               const gws_slm *slm, const gws_opts *opts, void *const *field_out);

/* Backward (MIXED only): given grad_field = dL/d(field) in PyTorch's complex convention
 * (dL/dRe + j dL/dIm), complex64 [n_lambda][H][W] (or dL/du_SLM with domain SPECTRUM),
 * writes dL/d(mean, quat, scale, opacity, amp) into out (device, same layout as the
 * inputs; every array is overwritten).  The spectra are recomputed, never stored.  In
 * SORTED_T mode the gradients include the cross terms through T_i = prod (1 - alpha_j(mu_i))
 * (Eq. 5-6 with Eq. 2; the set of factors above t_eps is held fixed). */
GWS_API gws_status gws_backward(const gws_gaussians *g, int64_t n, const gws_slm *slm, const gws_opts *opts,
                        const void *grad_field, gws_gaussians_grad *out);

/* Double-phase encoding: a = |u| / a_max (a_max = per-wavelength max |u|, or amp_scale if
 * > 0; a is clamped to 1), phi = arg u, P1,2 = phi -/+ acos(a); pixel (r, c) takes P1 when
 * r + c is even, else P2; wrapped to [-pi, pi).  field: complex64 (MIXED) or complex128
 * (FP64) [n_lambda][H][W]; phase_out: float [n_lambda][H][W]. */
GWS_API gws_status gws_encode(const void *field, const gws_slm *slm, const gws_opts *opts, float *phase_out,
                      float amp_scale);

/* Double-phase encoding for callers that cannot allocate device memory: code hosted inside
 * another application that owns every device allocation, or a real-time display loop that
 * fixes its memory at start-up and must not call cudaMalloc (which can synchronise the
 * device) mid-frame.  The paper has no counterpart; this is a deployment variant of
 * gws_encode with the same arguments and the same result.
 *   - opts->workspace is not used; prec selects complex64 / complex128 input as in gws_encode.
 *   - Its scratch (one slot per wavelength for the maximum amplitude) is a fixed array of
 *     GWS_NOALLOC_MAX_LAMBDA slots inside the library; every GPU that loads the library holds
 *     it until the process exits.  More wavelengths -> GWS_ERR_INVALID_ARG.
 *   - Each call made outside a stream capture looks up the array's device address on the
 *     current device (so a context rebuilt after cudaDeviceReset is served too) and remembers
 *     it; a call made while opts->stream is being captured uses the remembered address, so
 *     the first call on a device must come before any capture (else GWS_ERR_CUDA).
 *   - Argument checks are gws_encode's (same status for the same bad input), plus the limit
 *     below.
 *   - All calls share the array and each clears it before use: calls that overlap on the GPU
 *     (other streams, other host threads) race and must be serialised by the caller.
 *   - Calls no cudaMalloc, cudaFree or allocating library routine. */
#define GWS_NOALLOC_MAX_LAMBDA 16
GWS_API gws_status gws_encode_noalloc(const void *field, const gws_slm *slm, const gws_opts *opts, float *phase_out,
                                      float amp_scale);

/* Synchronises opts->stream and returns the device status word of the last call that
 * used this workspace (GWS_OK, GWS_ERR_NONFINITE, GWS_ERR_INVALID_ARG, GWS_ERR_TIMEOUT),
 * then clears it. */
GWS_API gws_status gws_get_device_status(const gws_opts *opts);

/* ---- inspection entry points (intermediate results of the forward, for testing) ---- */

/* Depth order (Algorithm S2: front = nearest the SLM = smallest mu_z; ties by index):
 * order_out[k] = input index of the k-th Gaussian, int32 device [n]. */
GWS_API gws_status gws_depth_order(const gws_gaussians *g, int64_t n, const gws_opts *opts, int32_t *order_out);

/* Transmittance T_i at each Gaussian's centre (SORTED_T reading of Eq. 5-6), FP64 device
 * [n], indexed by input order. */
GWS_API gws_status gws_transmittance(const gws_gaussians *g, int64_t n, const gws_opts *opts, double *T_out);

/* Spectral footprints of the MIXED path for wavelength index l: per input Gaussian the
 * normalised ellipse (a00, a01, a11) such that every frequency with fx^2 a00 + 2 fx fy a01
 * + fy^2 a11 > 1 has exp(-E) < trunc_eps; float device [n][3]. */
GWS_API gws_status gws_footprints(const gws_gaussians *g, int64_t n, const gws_slm *slm, const gws_opts *opts, int l,
                          float *ellipse_out);

/* Milliseconds between the events of timer `which` recorded by the last call on this host
 * thread that set GWS_DEBUG_TIME_KERNELS (synchronises on the stop event); -1 if none. */
GWS_API float gws_kernel_time_ms(int which);

/* Algorithmic work of the MIXED splat: the number of (Gaussian, wavelength, grid frequency)
 * triples inside the footprint ellipses (the pairs the truncated sum of Eq. 12 needs),
 * written to *pairs (host).  Synchronises the stream. */
GWS_API gws_status gws_footprint_pairs(const gws_gaussians *g, int64_t n, const gws_slm *slm, const gws_opts *opts,
                                       unsigned long long *pairs);

/* Number of kernel launches the last forward / backward / encode issued (host counter). */
GWS_API int gws_last_launch_count(void);

/* Autotuner of the MIXED splat: runs each splat configuration (gws_tile_config lists them:
 * frequency tile shape per CTA, pixels per thread, records per iteration, Gaussian records
 * per bulk-copied chunk, ring depth, CTAs per SM) twice on this scene with field_scratch
 * (complex64 [n_lambda][H][W]) as output, times the splat with CUDA events, and keeps the
 * fastest for this (H, W, n_lambda) in an in-process table used whenever opts.tile_cfg == 0.
 * Returns its id in *best_cfg.  Synchronises the stream; not capturable. */
/* The splat configurations the autotuner searches (no counterpart in the paper; the benchmark spec's
 * "tile shape and Gaussians per block").  Returns their number; for 1 <= id <= that number and
 * desc != NULL writes desc[0..7] = tile width, tile height (frequencies), pixels per thread,
 * records evaluated per iteration, Gaussian records per chunk, ring stages, CTAs per SM, pixel
 * pairs per thread whose cos runs on the FP32 pipe.  Host only. */
GWS_API int gws_tile_config(int id, int *desc);

/* gws_tile_config with the whole description (no counterpart in the paper, like
 * gws_tile_config): writes desc[0 .. min(n_desc, 9) - 1], the eight
 * values above followed by desc[8] = 1 where the configuration evaluates every second pixel
 * pair by the column step (its phase factor as the left neighbour's times one per-record
 * rotation and a first-order residual; chunks whose residual would exceed 2e-3 rad fall back
 * to the direct evaluation), else 0.  Host only. */
GWS_API int gws_tile_config_ext(int id, int *desc, int n_desc);

GWS_API gws_status gws_autotune(const gws_gaussians *g, int64_t n, const gws_slm *slm, const gws_opts *opts,
                        void *field_scratch, int *best_cfg);

/* The autotuner's in-process table (no counterpart in the paper), for callers that keep its
 * choices between processes.  gws_tune_get writes to *cfg (host) the configuration recorded for
 * slm's grid class (H, W, n_lambda) by gws_autotune or gws_tune_set, or 0 if there is none.
 * gws_tune_set records cfg (1 .. gws_tile_config(0, NULL)) for that class, as gws_autotune does
 * after timing, or forgets the class's entry for cfg = 0; other values give
 * GWS_ERR_INVALID_ARG.  Both check slm as gws_forward does, touch no device and are thread-safe. */
GWS_API gws_status gws_tune_get(const gws_slm *slm, int *cfg);
GWS_API gws_status gws_tune_set(const gws_slm *slm, int cfg);

/* ---- triangle primitive (supplement, polygon-based methods) ----------------------------------
 *
 * Eq. 10 with the canonical Gaussian replaced by the canonical triangle {(0,0), (1,0), (1,1)}:
 * for vertices v1, v2, v3 (hologram space), r1 = unit(v2 - v1), r3 = unit((v2 - v1) x (v3 - v1)),
 * r2 = r3 x r1, V_o = [[r1.(v2-v1), r1.(v3-v1)], [0, r2.(v3-v1)]], A = [[1,1],[0,1]] V_o^-1 and
 *   u_hat(f) = c o |r3 . f| / f_z |det V_o| T(A^-T (r1 . d, r2 . d)) e^{-j 2 pi f . v1}
 * (the affine theorem of Eq. 8; d = f - f_r, the on-axis reference wave of Sec. 4.1; T the
 * canonical triangle's spectrum; phase matching multiplies by e^{+j 2 pi v1_z / lambda}),
 * summed over triangles as in Eq. 12.  Every (triangle, frequency) pair is evaluated (the
 * spectrum of a triangle has no compact footprint). */
typedef struct { /* device memory */
    const double *vertices; /* [n][3][3]: v1, v2, v3, metres */
    const float *opacity;   /* [n] */
    const float *amp;       /* [n][n_lambda] */
} gws_triangles;

/* Workspace bytes for gws_forward_triangles with n triangles (opts.prec must be MIXED). */
GWS_API gws_status gws_triangles_workspace_size(int64_t n, const gws_slm *slm, const gws_opts *opts, size_t *bytes);

/* The field (or, with GWS_DOMAIN_SPECTRUM, the spectrum) of n triangles, complex64
 * [n_lambda][H][W] in field_out (device).  opts: prec MIXED (FP32 with FP64 per-(triangle, tile)
 * phase anchors), domain, phase_match, stream, workspace, GWS_DEBUG_TIME_KERNELS (the splat under
 * GWS_TIMER_SPLAT_FWD); blend is ignored.  A degenerate (zero-area) or non-finite triangle
 * contributes nothing and is recorded in the device status word (gws_get_device_status then
 * returns GWS_ERR_INVALID_ARG or GWS_ERR_NONFINITE).  Errors: GWS_ERR_INVALID_ARG,
 * GWS_ERR_UNSUPPORTED (FP64), GWS_ERR_WORKSPACE, GWS_ERR_CUDA. */
GWS_API gws_status gws_forward_triangles(const gws_triangles *t, int64_t n, const gws_slm *slm, const gws_opts *opts,
                                         void *field_out);

/* ---- holographics front end (Supplement Sec. 1.1) and view-dependent opacity (Sec. 4.2) ----
 *
 * Turns Gaussians optimised in world space (e.g. by a 2DGS / 2DGS-OIT model) into the
 * hologram-space inputs of the splat for one view:
 *   model transform   Sigma_w = R_w S_w S_w^T R_w^T                      (3 scales; surfel: s_z = 0)
 *   view transform    x_v = W x_w + t, the camera looking down -z
 *   projective map    perspective phi(x, y, z) = (fx x / (-z) + cx, fy y / (-z) + cy),
 *                     orthographic (fx x + cx, fy y + cy); J = d phi / dx at the mean (EWA)
 *   lifting           J W Sigma_w W^T J^T = R' S'^2 R'^T -> R_v = diag(R', 1), S_v = [S'; 0],
 *                     mu_v = (phi(W mu_w + t), (W mu_w + t)_z)
 *   hologram map      mu = A mu_v + b, Sigma = A R_v S_v S_v^T R_v^T A^T = R diag(s_u^2, s_v^2, 0) R^T
 * and the opacity factor SH(o, d) of alpha = G * SH(o, d): real spherical harmonics of degree
 * <= 3 (Condon-Shortley phase, m = -l..l), d the unit direction from the camera centre
 * -W^T t to mu_w, clamped to [0, 1].  The output scales are descending (s_u >= s_v), r3 =
 * r1 x r2 and the quaternion has w >= 0. */
typedef enum { GWS_PROJ_PERSPECTIVE = 0, GWS_PROJ_ORTHOGRAPHIC = 1 } gws_projection;

typedef struct { /* device memory */
    const double *mean;       /* [n][3] world-space means */
    const float *quat;        /* [n][4] world rotation (w, x, y, z), any non-zero norm */
    const float *scale;       /* [n][3] world scales (>= 0; a 2D surfel has scale[2] = 0) */
    const float *sh_opacity;  /* [n][sh_stride] SH coefficients of the opacity, or NULL */
    const float *opacity;     /* [n] view-independent opacity, used when sh_opacity is NULL */
    int sh_degree;            /* 0 .. 3: (sh_degree + 1)^2 coefficients are read */
    int sh_stride;            /* floats per Gaussian in sh_opacity; 0 means (sh_degree + 1)^2 */
} gws_world_gaussians;

typedef struct { /* writable Gaussians, same layout as gws_gaussians, device memory */
    double *mean;
    float *quat;
    float *scale;
    float *opacity;
    float *amp;
} gws_gaussians_out;

typedef struct { /* host values */
    double view[12];          /* row-major 3x4 [W | t]: x_view = W x_world + t */
    double fx, fy, cx, cy;    /* projective mapping into ray space */
    int projection;           /* gws_projection */
    double z_near;            /* a Gaussian is culled when its view depth -z is below z_near */
} gws_camera;

/* Front end for one view.  in: n world-space Gaussians (device).  cam: the view (host).
 * holo: HOST row-major 3x4 [A | b], ray space -> hologram space; A's first two columns must be
 * linearly independent.  Writes out->mean, out->quat, out->scale and out->opacity (device,
 * n entries each; out->amp is not touched and may be NULL) and, when valid is not NULL,
 * valid[i] = 1 for a kept Gaussian, 0 for a culled one (view depth below z_near, or a
 * non-finite / zero-norm input): culled entries get a zero mean, scales and opacity and the
 * identity rotation, and are meant to be dropped before the splat.  Runs on opts.stream
 * (other opts fields are ignored; no workspace).  Errors: GWS_ERR_INVALID_ARG for NULL
 * pointers (n > 0), n < 0, sh_degree outside 0..3, sh_stride below the coefficient count, an
 * unknown projection, non-finite camera / transform values or a rank-deficient A. */
GWS_API gws_status gws_holographics(const gws_world_gaussians *in, int64_t n, const gws_camera *cam,
                                    const double holo[12], const gws_opts *opts, gws_gaussians_out *out,
                                    unsigned char *valid);

#ifdef __cplusplus
}
#endif

#endif /* GWS_H */
