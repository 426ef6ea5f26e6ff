// gws_host.h -- internal host-side declarations shared by the libgws translation units.
#pragma once

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>
#include <stddef.h>
#include <stdint.h>

#include "gws_common.cuh"

namespace gws {

// NVTX range over the host-side enqueueing of one stage of a call (named in profiler
// timelines and usable as an ncu/nsys --nvtx filter; a no-op unless a tool is attached).
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange &) = delete;
    NvtxRange &operator=(const NvtxRange &) = delete;
};

// kernel-launch counter (gws_last_launch_count)
void count_launches(int k);

size_t sort_hist_words(long long n);

template <typename K>
cudaError_t radix_sort(K *&keys, K *&keys_alt, unsigned *&vals, unsigned *&vals_alt, long long n, int begin_bit,
                       int end_bit, unsigned *hist, cudaStream_t s, int *status = nullptr);

// ---- splat (forward) --------------------------------------------------------------------

struct Segs {
    int n_scenes;
    int n_lambda;
    long long off[GWS_MAX_SCENES + 1];  // Gaussian offsets of the scenes (concatenated)
};

// record range of segment (scene s, wavelength l): [L off[s] + l N_s, + N_s)
__host__ __device__ inline long long seg_start(const Segs &S, int seg) {
    int s = seg / S.n_lambda, l = seg % S.n_lambda;
    long long ns = S.off[s + 1] - S.off[s];
    return (long long)S.n_lambda * S.off[s] + (long long)l * ns;
}
__host__ __device__ inline long long seg_size(const Segs &S, int seg) {
    int s = seg / S.n_lambda;
    return S.off[s + 1] - S.off[s];
}

struct TileCfg {
    int id, tw, th;   // configuration id, frequency tile width x height per CTA
    int px, ru;       // pixels per thread, records evaluated per iteration
    int chunk, stages, ctas;  // Gaussian records per bulk-copied chunk, ring depth, CTAs per SM
    int npoly;        // pixel pairs per thread whose cos runs on the FP32 pipe (the rest on the MUFU)
    int step;         // 1: the odd pixel pairs by the column step (sin/cos of the even pairs rotated)
};
int n_tile_cfgs();
TileCfg tile_cfg(int id);  // id 1..n_tile_cfgs()

struct SplatArgs {
    const Rec *rec;
    const unsigned *items;   // item ids in processing order
    const int *item_count;   // records per item (prefix of the segment's footprint order)
    int n_items;
    int *queue;
    int *status;
    Segs segs;
    int H, W, tiles_x, n_tiles;
    double dfx, dfy;
    double inv_lam[GWS_MAX_LAMBDA];
    float dzmax[GWS_MAX_LAMBDA];  // the grid-wide |d_z| bound the records' footprints were built for
    int field_mode;  // 1: multiply by the centred-DFT pre-modulation
    int phase_match;
    unsigned long long timeout;
    unsigned debug;
    const float2 *pixtab;  // [lambda][H][W]: (f_z - f0_z of the pixel's tile, log2(1/f_z)) for these tiles
    void *out[GWS_MAX_SCENES];
};

cudaError_t launch_splat_mixed(int cfg, const SplatArgs &a, int grid, cudaStream_t s);
cudaError_t prepare_splat_kernels();
cudaError_t prepare_bwd_kernels();
int splat_mixed_ctas_per_sm(int cfg);

struct Splat64Args {
    const Rec64 *rec;
    const double *w;  // [n][n_lambda], depth-sorted order
    Segs segs;
    int H, W;
    double dfx, dfy;
    double inv_lam[GWS_MAX_LAMBDA];
    int field_mode;
    int phase_match;
    int *status;
    void *out[GWS_MAX_SCENES];
};
cudaError_t launch_splat_fp64(const Splat64Args &a, cudaStream_t s);

// ---- backward ---------------------------------------------------------------------------

struct BwdArgs {
    const Rec *rec;         // backward records (r3 unit, W separate), segment-major (single scene)
    const float4 *tab;      // (f_z - f0_z of the pixel's tile, log2 f_z - log2 |dL/du_SLM|), tile-major column pairs
    const float2 *ps;       // -arg dL/du_SLM, tile-major column pairs
    double *acc;            // [n_records][13] totals
    int *queue;
    int *status;
    Segs segs;
    int H, W, tiles_x, tiles_y;
    double dfx, dfy;
    double inv_lam[GWS_MAX_LAMBDA];
    float dzmax[GWS_MAX_LAMBDA];  // the grid-wide |d_z| bound the records' footprints were built for
    int phase_match;
    int n_items;            // (wavelength, block of records) work items
};

struct GradArgs {
    double *mean;
    float *quat, *scale, *opacity, *amp;
    double *dT;             // optional dL/dT_i (depth-sorted mode)
    int *status;            // device status word (index checks of the checking build)
    int phase_match;
    double inv_lam[GWS_MAX_LAMBDA];
};

struct InvLam {
    double v[GWS_MAX_LAMBDA];
};

cudaError_t launch_pixtab(int n_lambda, int H, int W, double dfx, double dfy, const InvLam &il, int tw, int th,
                          float2 *tab, cudaStream_t s);

// ---- triangle primitive ------------------------------------------------------------------

struct TriRec {     // 64 B per triangle
    double v1[3];   // first vertex (the translation)
    float M[6];     // rows of A^-T [r1; r2]: nu = M d, d = f - f_r
    float r3[3];    // unit normal
    float pad;
};
cudaError_t launch_tri_prep(const double *v, const float *opacity, const float *amp, long long n, int L, TriRec *rec,
                            float *w, int *status, cudaStream_t s);
cudaError_t launch_splat_tri(const TriRec *rec, const float *w, long long n, int L, int H, int W, double dfx,
                             double dfy, const InvLam &il, int field_mode, int phase_match, float2 *out,
                             cudaStream_t s);
cudaError_t launch_splat_bwd(const BwdArgs &a, int grid, cudaStream_t s);
cudaError_t launch_grad_assemble(const GPre *gp, const float *ampc, const double *T_g, const int *invrec,
                                 const double *acc, const float *quat_in, long long n, int L, const GradArgs &G,
                                 cudaStream_t s);
int bwd_block_size();
int bwd_ctas_per_sm();
int bwd_tiles_x(int W);
int bwd_tiles_y(int H);
size_t bwd_table_bytes(int n_lambda, int H, int W);  // one float4 tile-major table (the float2 one takes half)
cudaError_t launch_bwd_tables(int n_lambda, int H, int W, double dfx, double dfy, const InvLam &il, const float2 *G,
                              float4 *tab, float2 *ps, cudaStream_t s);

}  // namespace gws
