// gws_prep.h -- host launchers of the non-splat kernels (gws_prep.cu).
#pragma once

#include "gws_host.h"

namespace gws {

struct FootParams {
    float rho;                     // sqrt(ln(1/eps) / (2 pi^2))
    float dzmax[GWS_MAX_LAMBDA];   // max |f_z - 1/lambda| over the grid, per wavelength
};

cudaError_t launch_prep(const SceneTable &T, long long n_total, GPre *gp, float *ampc, unsigned long long *dkey,
                        unsigned *dval, int *status, cudaStream_t s);
cudaError_t launch_scene_key(const GPre *gp, const unsigned *sorted, long long n, unsigned *skey, cudaStream_t s);
cudaError_t launch_transmittance(const GPre *gp, const unsigned *sorted, const Segs &S, long long n, double alpha_min,
                                 TData *td, double *T_sorted, double *T_g, TQuery *tq, cudaStream_t s);
cudaError_t launch_tgrad(const TData *td, TQuery *tq, const GPre *gp, const unsigned *sorted, const double *dT_g,
                         const float *quat_in, const Segs &S, long long n, double alpha_min, double *dmean,
                         float *dquat, float *dscale, float *dopacity, cudaStream_t s);
cudaError_t launch_rec64(const GPre *gp, const float *ampc, const unsigned *sorted, const double *T_sorted, long long n,
                         int L, Rec64 *rec, double *w, cudaStream_t s);
cudaError_t launch_foot_keys(const GPre *gp, const float *ampc, const unsigned *sorted, const double *T_sorted,
                             const Segs &S, long long n_rec, const FootParams &F, int drop_zero,
                             unsigned long long *key, unsigned *val, cudaStream_t s);
cudaError_t launch_gather(const unsigned long long *key, const unsigned *val, const GPre *gp, const float *ampc,
                          const unsigned *sorted, const double *T_sorted, const Segs &S, long long n_rec,
                          const FootParams &F, int drop_zero, int backward, Rec *rec, float *Rr, int *invrec,
                          int *status, cudaStream_t s);
cudaError_t launch_foot_inspect(const GPre *gp, long long n, float rho, float dzmax, float *out, cudaStream_t s);
cudaError_t launch_items(const float *Rr, const Segs &S, int n_seg, int H, int W, int tw, int th, int tiles_x,
                         int n_tiles, double dfx, double dfy, unsigned long long *ikey, unsigned *ival, int *icount,
                         cudaStream_t s);
cudaError_t launch_count_pairs(const GPre *gp, long long n, int n_lambda, const FootParams &F, int H, int W,
                               double dfx, double dfy, unsigned long long *acc, cudaStream_t s);
cudaError_t launch_modulate(void *data, int prec64, int n_slices, int H, int W, double scale, int mode,
                            cudaStream_t s);
struct ExactBatch {  // one batch of exact blending (Gaussians in depth order)
    double *mean;    // [B][3], depth component zeroed
    float *quat;     // [B][4]
    float *scale;    // [B][2]
    float *opacity;  // [B] (1: the field itself)
    float *amp;      // [B][L] (1)
    double *zk;      // [B] depths
    float *co;       // [B][L] c o
    float *ok;       // [B] o
    double *mu;      // [B][3] the means (partial coherence: the inner fields sit at the origin)
    float *rr;       // [B][9] kappa s_u r1, kappa s_v r2, 2 pi s_u s_v r3 (the one-Gaussian record)
    int *status;     // device status word (index checks of the checking build)
    long long n;     // Gaussians of the scene (bound of the depth-order indices)
};
// pc = 0: exact blending (the means keep x, y; depth zeroed); pc = 1: partial coherence (means zeroed)
cudaError_t launch_exact_gather(const unsigned *sorted, long long b0, int nb, const gws_gaussians *g, int L,
                                const ExactBatch &E, int pc, cudaStream_t s);
// partial coherence: the angular kernel K [L][H][W] (FP32 complex) and sum_f Y^2 per wavelength
// (accumulated into ysum, which must be zeroed first)
cudaError_t launch_pc_kernel(float2 *K, double *ysum, int sh_l, int sh_m, unsigned long long seed,
                             unsigned long long frame, int L, int H, int W, double dfx, double dfy,
                             const InvLam &il, cudaStream_t s);
// w_k = c_k o_k u_k kappa / sqrt(ysum) for the batch's fields [nb][L][H][W], from Uin into Uout
// (the same buffer for one frame; another when several frames share the batch's fields)
cudaError_t launch_pc_apply(const float2 *Uin, float2 *Uout, const float2 *kappa, const double *ysum,
                            const ExactBatch &E, int nb, int L, long long hw, float uscale, cudaStream_t s);
// the batch's one-Gaussian spectra (Eq. 10, c = o = T = 1, dense) with the centred pre-modulation,
// U [nb][L][H][W]; pixtab: the natural-layout table for 64 x 32 tiles
cudaError_t launch_single_spectra(const ExactBatch &E, int nb, int L, int H, int W, double dfx, double dfy,
                                  const InvLam &il, const float2 *pixtab, float2 *U, cudaStream_t s);
// acc += sum_k V_k(f) e^{-j 2 pi f . mu_k} (x e^{+j 2 pi mu_z / lambda} with phase matching)
cudaError_t launch_pc_accum(const float2 *V, float2 *acc, const float2 *pixtab, const ExactBatch &E, int nb, int L,
                            int H, int W, double dfx, double dfy, const InvLam &il, int phase_match, int fold,
                            float vscale, cudaStream_t s);
cudaError_t launch_fill(float *p, long long n, float v, cudaStream_t s);
cudaError_t launch_exact_mask(float2 *U, float *T, const ExactBatch &E, int nb, int L, long long hw, float t_eps,
                              float t_bin, float uscale, cudaStream_t s);
cudaError_t launch_exact_accum(const float2 *V, float2 *acc, const float2 *pixtab, const ExactBatch &E, int nb, int L,
                               int H, int W, double dfx, double dfy, const InvLam &il, int fold, float vscale,
                               cudaStream_t s);

cudaError_t launch_encode(const void *field, int prec64, int n_lambda, int H, int W, unsigned long long *amax2,
                          double amp_scale, float *out, cudaStream_t s);
// argument checks of the encoding (grid, options, pointers, finite amp_scale), shared by
// gws_encode and gws_encode_noalloc so that both return the same status for the same input
gws_status check_encode_args(const void *field, const gws_slm *slm, const gws_opts *opts, const float *phase_out,
                             float amp_scale);

}  // namespace gws
