// gws_api.cu -- the C ABI of libgws (declared in include/gws.h): argument checks, the
// workspace layout, the cuFFT plan cache and the launch sequence of each entry point.
#include <cufft.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include "gws_prep.h"

namespace gws {

static thread_local int t_launches = 0;
void count_launches(int k) { t_launches += k; }

// ---- optional kernel timers (GWS_DEBUG_TIME_KERNELS) -----------------------------------
struct Timers {
    cudaEvent_t ev[5][2];
    bool made = false, used[5] = {false, false, false, false, false};
};
static thread_local Timers t_timers;

static void timer_mark(const gws_opts *o, int which, int edge, cudaStream_t s) {
    if (!(o->debug_flags & GWS_DEBUG_TIME_KERNELS)) return;
    Timers &T = t_timers;
    if (!T.made) {
        for (int i = 0; i < 5; ++i)
            for (int j = 0; j < 2; ++j) cudaEventCreate(&T.ev[i][j]);
        T.made = true;
    }
    cudaEventRecord(T.ev[which][edge], s);
    if (edge == 1) T.used[which] = true;
}
static void timers_reset(const gws_opts *o) {
    if (!(o->debug_flags & GWS_DEBUG_TIME_KERNELS)) return;
    for (int i = 0; i < 5; ++i) t_timers.used[i] = false;
}

// cuFFT batch size of one scene's slices
struct PlanKey {
    int dev, H, W, batch, dbl, dir;
    bool operator<(const PlanKey &o) const {
        return std::tie(dev, H, W, batch, dbl, dir) < std::tie(o.dev, o.H, o.W, o.batch, o.dbl, o.dir);
    }
};
struct Plan {
    cufftHandle h;
    size_t work;
};
static std::mutex g_plan_mu;
static std::map<PlanKey, Plan> g_plans;

static gws_status get_plan(int H, int W, int batch, int dbl, Plan *out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return GWS_ERR_CUDA;
    std::lock_guard<std::mutex> lk(g_plan_mu);
    PlanKey k{dev, H, W, batch, dbl, 0};
    auto it = g_plans.find(k);
    if (it != g_plans.end()) {
        *out = it->second;
        return GWS_OK;
    }
    Plan p;
    if (cufftCreate(&p.h) != CUFFT_SUCCESS) return GWS_ERR_CUDA;
    if (cufftSetAutoAllocation(p.h, 0) != CUFFT_SUCCESS) return GWS_ERR_CUDA;
    int dims[2] = {H, W};
    size_t work = 0;
    cufftResult r = cufftMakePlanMany(p.h, 2, dims, nullptr, 1, H * W, nullptr, 1, H * W, dbl ? CUFFT_Z2Z : CUFFT_C2C,
                                      batch, &work);
    if (r != CUFFT_SUCCESS) {
        cufftDestroy(p.h);
        return GWS_ERR_CUDA;
    }
    p.work = work;
    g_plans[k] = p;
    *out = p;
    return GWS_OK;
}

// a plan that already exists (no creation in the call path)
static bool cached_plan(int H, int W, int batch, int dbl, Plan *out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return false;
    std::lock_guard<std::mutex> lk(g_plan_mu);
    auto it = g_plans.find(PlanKey{dev, H, W, batch, dbl, 0});
    if (it == g_plans.end()) return false;
    *out = it->second;
    return true;
}

static gws_status exec_fft(const Plan &p, void *data, void *work, int dbl, int direction, cudaStream_t s) {
    std::lock_guard<std::mutex> lk(g_plan_mu);
    if (cufftSetStream(p.h, s) != CUFFT_SUCCESS) return GWS_ERR_CUDA;
    if (cufftSetWorkArea(p.h, work) != CUFFT_SUCCESS) return GWS_ERR_CUDA;
    cufftResult r = dbl ? cufftExecZ2Z(p.h, (cufftDoubleComplex *)data, (cufftDoubleComplex *)data, direction)
                        : cufftExecC2C(p.h, (cufftComplex *)data, (cufftComplex *)data, direction);
    count_launches(1);
    return r == CUFFT_SUCCESS ? GWS_OK : GWS_ERR_CUDA;
}

// ---------------------------------------------------------------------------------------
// workspace layout (one planner for the size query and for the calls)
// ---------------------------------------------------------------------------------------

#ifdef GWS_CHECK_BOUNDS
// checking build: 64 bytes of canary words after every workspace sub-buffer
constexpr size_t kCanaryBytes = 64;
constexpr int kMaxCanaries = 64;
#endif

struct Layout {
#ifdef GWS_CHECK_BOUNDS
    size_t canary[kMaxCanaries];
    int n_canary;
#endif
    size_t status, queue, amax, gpre, ampc, dkey0, dkey1, dval0, dval1, skey0, skey1, hist, tsorted, tg, tdata;
    size_t rec64, w64, fkey0, fkey1, fval0, fval1, rec, Rr, ikey0, ikey1, ival0, ival1, icount, invrec, gspec, bacc;
    size_t pixtab, gtiles, dT, tq;
    size_t ex_U, ex_T, ex_arr;
    size_t pc_kappa, pc_ysum;  // partial coherence: the kernel patterns [F][L][H][W] and sum_f Y^2 [F][L]
    size_t ex_U2;              // partial coherence over F > 1 frames: one frame's copy of the batch's fields
    int ex_B;
    size_t cufft, total;
    int tiles_x, tiles_y, n_tiles, cfg;
};

static size_t align_up(size_t x) { return (x + 255) & ~(size_t)255; }

struct Planner {
    size_t cur = 0;
#ifdef GWS_CHECK_BOUNDS
    size_t canary[kMaxCanaries];
    int n_canary = 0;
    size_t take(size_t bytes) {
        // the canary starts right after the buffer (16-byte granularity), then the usual alignment
        const size_t o = cur;
        const size_t end = o + ((std::max<size_t>(bytes, 16) + 15) & ~(size_t)15);
        if (n_canary < kMaxCanaries) canary[n_canary++] = end;
        cur = align_up(end + kCanaryBytes);
        return o;
    }
#else
    size_t take(size_t bytes) {
        size_t o = cur;
        cur = align_up(cur + std::max<size_t>(bytes, 16));
        return o;
    }
#endif
};

// tile configuration chosen by gws_autotune per grid class (H, W, n_lambda)
static std::mutex g_tune_mu;
static std::map<std::tuple<int, int, int>, int> g_tuned;

static int default_cfg(const gws_opts *o, const gws_slm *slm) {
    int c = o->tile_cfg;
    if (c >= 1 && c <= n_tile_cfgs()) return c;
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tuned.find(std::make_tuple(slm->H, slm->W, slm->n_lambda));
    return it != g_tuned.end() ? it->second : 1;
}

static int pc_frames(const gws_opts *o) { return o->pc_frames > 1 ? o->pc_frames : 1; }

static int exact_batch(const gws_opts *o) {
    int B = o->exact_batch > 0 ? o->exact_batch : 128;
    return B > GWS_MAX_SCENES ? GWS_MAX_SCENES : B;
}

static gws_status plan_layout(long long n_total, int n_scenes, const gws_slm *slm, const gws_opts *o, Layout *L,
                              bool need_fft_plans) {
    Planner P;
    const int nl = slm->n_lambda;
    const long long n = std::max<long long>(n_total, 1);
    const long long n_rec = n * nl;
    L->cfg = default_cfg(o, slm);
    const TileCfg tc = tile_cfg(L->cfg);
    L->tiles_x = (slm->W + tc.tw - 1) / tc.tw;
    L->tiles_y = (slm->H + tc.th - 1) / tc.th;
    L->n_tiles = L->tiles_x * L->tiles_y;
    // item arrays sized for the configuration with the most tiles, so that a later tuning
    // never outgrows a workspace sized earlier
    long long max_tiles = 0;
    for (int c = 1; c <= n_tile_cfgs(); ++c) {
        const TileCfg t = tile_cfg(c);
        max_tiles = std::max(max_tiles, (long long)((slm->W + t.tw - 1) / t.tw) * ((slm->H + t.th - 1) / t.th));
    }
    const long long n_items = (long long)n_scenes * nl * max_tiles;

    L->status = P.take(16);
    L->queue = P.take(16);
    L->amax = P.take(sizeof(unsigned long long) * GWS_MAX_LAMBDA);
    L->gpre = P.take(sizeof(GPre) * n);
    L->ampc = P.take(sizeof(float) * n * nl);
    L->dkey0 = P.take(8 * n);
    L->dkey1 = P.take(8 * n);
    L->dval0 = P.take(4 * n);
    L->dval1 = P.take(4 * n);
    L->skey0 = P.take(4 * n);
    L->skey1 = P.take(4 * n);
    L->tsorted = P.take(8 * n);
    L->tg = P.take(8 * n);
    L->tdata = P.take(sizeof(TData) * n);
    L->tq = P.take(sizeof(TQuery) * n);
    size_t hist_words = std::max(sort_hist_words(n), sort_hist_words(std::max(n_rec, n_items)));
    L->hist = P.take(4 * hist_words);
    if (o->prec == GWS_PREC_FP64) {
        L->rec64 = P.take(sizeof(Rec64) * n);
        L->w64 = P.take(8 * n * nl);
        L->fkey0 = L->fkey1 = L->fval0 = L->fval1 = L->rec = L->Rr = 0;
        L->ikey0 = L->ikey1 = L->ival0 = L->ival1 = L->icount = L->invrec = L->gspec = L->bacc = 0;
        L->pixtab = L->gtiles = L->dT = 0;
    } else {
        L->rec64 = L->w64 = 0;
        L->fkey0 = P.take(8 * n_rec);
        L->fkey1 = P.take(8 * n_rec);
        L->fval0 = P.take(4 * n_rec);
        L->fval1 = P.take(4 * n_rec);
        L->rec = P.take(sizeof(Rec) * n_rec);
        L->Rr = P.take(4 * n_rec);
        L->ikey0 = P.take(8 * n_items);
        L->ikey1 = P.take(8 * n_items);
        L->ival0 = P.take(4 * n_items);
        L->ival1 = P.take(4 * n_items);
        L->icount = P.take(4 * n_items);
        L->invrec = P.take(4 * n_rec);
        L->gspec = P.take(sizeof(float) * 2 * (size_t)nl * slm->H * slm->W);
        L->bacc = P.take(sizeof(double) * 13 * n_rec);
        // the backward's tile-major tables (also the natural-layout table of the exact blend)
        L->pixtab = P.take(std::max(bwd_table_bytes(nl, slm->H, slm->W), sizeof(float) * 2 * (size_t)nl * slm->H * slm->W));
        L->gtiles = P.take(bwd_table_bytes(nl, slm->H, slm->W));
        L->dT = P.take(sizeof(double) * n);
    }
    L->ex_U = L->ex_T = L->ex_arr = 0;
    L->pc_kappa = L->pc_ysum = L->ex_U2 = 0;
    L->ex_B = 0;
    size_t fft_work = 0;
    const bool pc = o->blend == GWS_BLEND_PARTIAL_COHERENT;
    if ((o->blend == GWS_BLEND_EXACT || pc) && o->prec == GWS_PREC_MIXED) {
        const int B = exact_batch(o);
        L->ex_B = B;
        const size_t hw = (size_t)slm->H * slm->W;
        L->ex_U = P.take(sizeof(float) * 2 * (size_t)B * nl * hw);
        if (pc) {
            const size_t nf = (size_t)pc_frames(o);
            L->pc_kappa = P.take(sizeof(float) * 2 * nf * nl * hw);
            L->pc_ysum = P.take(sizeof(double) * nf * nl);
            if (nf > 1) L->ex_U2 = P.take(sizeof(float) * 2 * (size_t)B * nl * hw);
        } else {
            L->ex_T = P.take(sizeof(float) * nl * hw);
        }
        L->ex_arr = P.take((size_t)B * (24 + 16 + 8 + 4 + 4 * nl + 8 + 4 * nl + 4 + 24 + 36) + 256 * 10);
        Plan p;  // the batch path always transforms (each batch's fields both ways, the final inverse)
        gws_status st = get_plan(slm->H, slm->W, nl, 0, &p);
        if (st != GWS_OK) return st;
        fft_work = std::max(fft_work, p.work);
        st = get_plan(slm->H, slm->W, B * nl, 0, &p);
        if (st != GWS_OK) return st;
        fft_work = std::max(fft_work, p.work);
    }
    if (need_fft_plans) {
        Plan p;
        gws_status st = get_plan(slm->H, slm->W, nl, o->prec == GWS_PREC_FP64, &p);
        if (st != GWS_OK) return st;
        fft_work = std::max(fft_work, p.work);
        if (n_scenes > 1) {  // one batched transform when the scenes' outputs are contiguous
            st = get_plan(slm->H, slm->W, n_scenes * nl, o->prec == GWS_PREC_FP64, &p);
            if (st != GWS_OK) return st;
            fft_work = std::max(fft_work, p.work);
        }
    }
    L->cufft = P.take(fft_work);
    L->total = P.cur;
#ifdef GWS_CHECK_BOUNDS
    L->n_canary = P.n_canary;
    for (int i = 0; i < P.n_canary; ++i) L->canary[i] = P.canary[i];
#endif
    return GWS_OK;
}

// Checking build: a call's workspace canaries are written when its guard is made (after the
// workspace checks) and verified when the guard goes out of scope (every return path), on the
// call's stream; an overwritten word sets ST_BOUNDS in the status word.  The product build's
// guard does nothing.
#ifdef GWS_CHECK_BOUNDS
struct CanaryList {
    int n;
    unsigned long long off[kMaxCanaries];
};
__global__ void k_canary(unsigned char *ws, CanaryList c, int check, int *status) {
    constexpr int words = (int)(kCanaryBytes / 4);
    for (int i = threadIdx.x; i < c.n * words; i += blockDim.x) {
        unsigned *w = reinterpret_cast<unsigned *>(ws + c.off[i / words]) + (i % words);
        const unsigned pat = 0xC0DE5A5Au ^ ((unsigned)i * 2654435761u);
        if (check) {
            if (*w != pat) atomicOr(status, ST_BOUNDS);
        } else {
            *w = pat;
        }
    }
}
struct CanaryGuard {
    const gws_opts *o;
    CanaryList c;
    size_t status;
    cudaStream_t s;
    template <class LayoutT>
    CanaryGuard(const gws_opts *o_, const LayoutT &L, cudaStream_t s_) : o(o_), status(L.status), s(s_) {
        c.n = L.n_canary;
        for (int i = 0; i < L.n_canary; ++i) c.off[i] = L.canary[i];
        k_canary<<<1, 256, 0, s>>>(static_cast<unsigned char *>(o->workspace), c, 0, nullptr);
    }
    ~CanaryGuard() {
        k_canary<<<1, 256, 0, s>>>(static_cast<unsigned char *>(o->workspace), c, 1,
                                   reinterpret_cast<int *>(static_cast<char *>(o->workspace) + status));
    }
};
#else
struct CanaryGuard {
    template <class LayoutT>
    CanaryGuard(const gws_opts *, const LayoutT &, cudaStream_t) {}
};
#endif

// ---------------------------------------------------------------------------------------
// argument checks
// ---------------------------------------------------------------------------------------

static bool finite_pos(double x) { return std::isfinite(x) && x > 0; }

static gws_status check_slm(const gws_slm *slm) {
    if (!slm) return GWS_ERR_INVALID_ARG;
    if (slm->H < 1 || slm->W < 1 || (long long)slm->H * slm->W > (1ll << 31)) return GWS_ERR_INVALID_ARG;
    if (!finite_pos(slm->pitch_x) || !finite_pos(slm->pitch_y)) return GWS_ERR_INVALID_ARG;
    if (slm->n_lambda < 1 || slm->n_lambda > GWS_MAX_LAMBDA || !slm->wavelengths) return GWS_ERR_INVALID_ARG;
    for (int l = 0; l < slm->n_lambda; ++l)
        if (!finite_pos(slm->wavelengths[l])) return GWS_ERR_INVALID_ARG;
    return GWS_OK;
}

static gws_status check_opts(const gws_opts *o) {
    if (!o) return GWS_ERR_INVALID_ARG;
    if (o->blend != GWS_BLEND_OIT && o->blend != GWS_BLEND_SORTED_T && o->blend != GWS_BLEND_EXACT &&
        o->blend != GWS_BLEND_PARTIAL_COHERENT)
        return GWS_ERR_INVALID_ARG;
    if (o->pc_l < 0 || o->pc_l > 3 || o->pc_m < -o->pc_l || o->pc_m > o->pc_l) return GWS_ERR_INVALID_ARG;
    if (o->pc_frames < 0 || o->pc_frames > GWS_MAX_PC_FRAMES) return GWS_ERR_INVALID_ARG;
    if (!(o->t_binarize >= 0.f && o->t_binarize < 1.f) || o->exact_batch < 0) return GWS_ERR_INVALID_ARG;
    if (o->prec != GWS_PREC_FP64 && o->prec != GWS_PREC_MIXED) return GWS_ERR_INVALID_ARG;
    if (o->domain != GWS_DOMAIN_FIELD && o->domain != GWS_DOMAIN_SPECTRUM) return GWS_ERR_INVALID_ARG;
    if (!(o->trunc_eps > 0.f && o->trunc_eps < 1.f)) return GWS_ERR_INVALID_ARG;
    if (!(o->alpha_min >= 0.f && o->alpha_min < 1.f)) return GWS_ERR_INVALID_ARG;
    if (o->timeout_cycles == 0) return GWS_ERR_INVALID_ARG;
    if (o->tile_cfg < 0 || o->tile_cfg > n_tile_cfgs()) return GWS_ERR_INVALID_ARG;
    return GWS_OK;
}

static gws_status check_gaussians(const gws_gaussians *g, long long n) {
    if (n < 0 || n > (1ll << 30)) return GWS_ERR_INVALID_ARG;
    if (n == 0) return GWS_OK;
    if (!g || !g->mean || !g->quat || !g->scale || !g->opacity || !g->amp) return GWS_ERR_INVALID_ARG;
    return GWS_OK;
}

static gws_status check_workspace(const gws_opts *o, const Layout &L) {
    if (!o->workspace) return GWS_ERR_WORKSPACE;
    if (((uintptr_t)o->workspace) & 255u) return GWS_ERR_WORKSPACE;
    if (o->workspace_bytes < L.total) return GWS_ERR_WORKSPACE;
    return GWS_OK;
}

#define CU(x)                                    \
    do {                                         \
        if ((x) != cudaSuccess) return GWS_ERR_CUDA; \
    } while (0)
#define GS(x)                          \
    do {                               \
        gws_status _s = (x);           \
        if (_s != GWS_OK) return _s;   \
    } while (0)

template <typename T>
static T *at(const gws_opts *o, size_t off) {
    return reinterpret_cast<T *>(static_cast<char *>(o->workspace) + off);
}

static double dz_max(const gws_slm *slm, double lam) {
    const double fxm = (double)(slm->W / 2) / (slm->W * slm->pitch_x);
    const double fym = (double)(slm->H / 2) / (slm->H * slm->pitch_y);
    const double rho2 = fxm * fxm + fym * fym, k2 = 1.0 / (lam * lam);
    return rho2 >= k2 ? 1.0 / lam : 1.0 / lam - std::sqrt(k2 - rho2);
}

// ---------------------------------------------------------------------------------------
// shared front half: validation, depth sort, transmittance
// ---------------------------------------------------------------------------------------

struct Front {
    SceneTable T;
    Segs S;
    long long n_total;
    unsigned *sorted;  // depth-sorted global indices
    double *T_sorted;  // null in OIT mode
    double *T_g;
};

static gws_status run_front(const gws_gaussians *scenes, const int64_t *n, int n_scenes, const gws_slm *slm,
                            const gws_opts *o, const Layout &L, bool need_T, Front *F, cudaStream_t s) {
    NvtxRange nvtx("gws: validate, depth sort, transmittance");
    SceneTable &T = F->T;
    std::memset(&T, 0, sizeof T);
    T.n_scenes = n_scenes;
    T.n_lambda = slm ? slm->n_lambda : 1;
    T.off[0] = 0;
    for (int k = 0; k < n_scenes; ++k) {
        T.off[k + 1] = T.off[k] + n[k];
        T.mean[k] = scenes[k].mean;
        T.quat[k] = scenes[k].quat;
        T.scale[k] = scenes[k].scale;
        T.opacity[k] = scenes[k].opacity;
        T.amp[k] = scenes[k].amp;
    }
    F->S.n_scenes = n_scenes;
    F->S.n_lambda = T.n_lambda;
    std::memcpy(F->S.off, T.off, sizeof(T.off));
    F->n_total = T.off[n_scenes];
    const long long nt = F->n_total;
    GPre *gp = at<GPre>(o, L.gpre);
    unsigned long long *dk0 = at<unsigned long long>(o, L.dkey0), *dk1 = at<unsigned long long>(o, L.dkey1);
    unsigned *dv0 = at<unsigned>(o, L.dval0), *dv1 = at<unsigned>(o, L.dval1);
    CU(launch_prep(T, nt, gp, at<float>(o, L.ampc), dk0, dv0, at<int>(o, L.status), s));
    unsigned *hist = at<unsigned>(o, L.hist);
    CU(radix_sort<unsigned long long>(dk0, dk1, dv0, dv1, nt, 0, 64, hist, s, at<int>(o, L.status)));
    if (n_scenes > 1) {
        unsigned *sk0 = at<unsigned>(o, L.skey0), *sk1 = at<unsigned>(o, L.skey1);
        CU(launch_scene_key(gp, dv0, nt, sk0, s));
        CU(radix_sort<unsigned>(sk0, sk1, dv0, dv1, nt, 0, 8, hist, s, at<int>(o, L.status)));
    }
    F->sorted = dv0;
    F->T_sorted = nullptr;
    F->T_g = nullptr;
    if (need_T) {
        F->T_sorted = at<double>(o, L.tsorted);
        F->T_g = at<double>(o, L.tg);
        CU(launch_transmittance(gp, dv0, F->S, nt, (double)o->alpha_min, at<TData>(o, L.tdata), F->T_sorted, F->T_g,
                                at<TQuery>(o, L.tq), s));
    }
    return GWS_OK;
}

static FootParams foot_params(const gws_slm *slm, const gws_opts *o) {
    FootParams F;
    std::memset(&F, 0, sizeof F);
    F.rho = (float)std::sqrt(std::log(1.0 / (double)o->trunc_eps) / (2.0 * kPi * kPi));
    for (int l = 0; l < slm->n_lambda; ++l) F.dzmax[l] = (float)(dz_max(slm, slm->wavelengths[l]) * 1.0001);
    return F;
}

static int seg_bits(int n_seg) {
    int b = 0;
    while ((1 << b) < n_seg) ++b;
    return ((b + 7) / 8) * 8;
}

// records in decreasing-footprint order per segment; returns the record array
static gws_status run_records(const Front &F, const gws_slm *slm, const gws_opts *o, const Layout &L, int backward,
                              cudaStream_t s, Rec **rec_out) {
    NvtxRange nvtx("gws: footprints, binning, records");
    const long long n_rec = F.n_total * slm->n_lambda;
    const FootParams FP = foot_params(slm, o);
    GPre *gp = at<GPre>(o, L.gpre);
    unsigned long long *k0 = at<unsigned long long>(o, L.fkey0), *k1 = at<unsigned long long>(o, L.fkey1);
    unsigned *v0 = at<unsigned>(o, L.fval0), *v1 = at<unsigned>(o, L.fval1);
    const int drop = backward ? 0 : 1;
    CU(launch_foot_keys(gp, at<float>(o, L.ampc), F.sorted, F.T_sorted, F.S, n_rec, FP, drop, k0, v0, s));
    const int n_seg = F.S.n_scenes * F.S.n_lambda;
    CU(radix_sort<unsigned long long>(k0, k1, v0, v1, n_rec, 0, 32 + seg_bits(n_seg), at<unsigned>(o, L.hist), s,
                                      at<int>(o, L.status)));
    Rec *rec = at<Rec>(o, L.rec);
    CU(launch_gather(k0, v0, gp, at<float>(o, L.ampc), F.sorted, F.T_sorted, F.S, n_rec, FP, drop, backward, rec,
                     at<float>(o, L.Rr), backward ? at<int>(o, L.invrec) : nullptr, at<int>(o, L.status), s));
    *rec_out = rec;
    return GWS_OK;
}

static int num_sms() {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return sms > 0 ? sms : 1;
}

static gws_status forward_impl(const gws_gaussians *scenes, const int64_t *n, int n_scenes, const gws_slm *slm,
                               const gws_opts *o, void *const *out);

// One FFT over nb slices of L [H][W] planes: the cached batched plan when the batch is full,
// else slice by slice.
static gws_status batch_fft(const Plan &p, int H, int W, int nl, int nb, int B, float2 *U, void *work, int dir,
                            cudaStream_t s) {
    Plan pb;
    if (nb == B && cached_plan(H, W, B * nl, 0, &pb)) return exec_fft(pb, U, work, 0, dir, s);
    const long long hw = (long long)H * W;
    for (int k = 0; k < nb; ++k) GS(exec_fft(p, U + (size_t)k * nl * hw, work, 0, dir, s));
    return GWS_OK;
}

// Exact alpha wave blending (Algorithm S2), front to back in batches of B Gaussians; see
// gws_exact.cu.  The batch's fields at their own planes: each Gaussian's dense spectrum (Eq. 10
// with the depth component of the mean zeroed, c = o = 1; k_single_spectra) and one batched
// inverse FFT.
static gws_status exact_forward(const gws_gaussians *scene, long long n, const gws_slm *slm, const gws_opts *o,
                                const Layout &L, const Front &F, void *out, cudaStream_t s) {
    NvtxRange nvtx("gws: exact blending");
    const int nl = slm->n_lambda, H = slm->H, W = slm->W;
    const long long hw = (long long)H * W;
    const double dfx = 1.0 / (W * slm->pitch_x), dfy = 1.0 / (H * slm->pitch_y);
    const int B = L.ex_B;
    float2 *acc = static_cast<float2 *>(out);
    float2 *U = at<float2>(o, L.ex_U);
    float *Tm = at<float>(o, L.ex_T);
    char *arr = at<char>(o, L.ex_arr);
    ExactBatch E;
    E.mean = reinterpret_cast<double *>(arr);
    E.zk = E.mean + 3 * B;
    E.quat = reinterpret_cast<float *>(E.zk + B);
    E.scale = E.quat + 4 * B;
    E.opacity = E.scale + 2 * B;
    E.amp = E.opacity + B;
    E.co = E.amp + (size_t)B * nl;
    E.ok = E.co + (size_t)B * nl;
    E.rr = E.ok + B;
    E.mu = nullptr;
    E.status = at<int>(o, L.status);
    E.n = n;
    InvLam il;
    std::memset(&il, 0, sizeof il);
    for (int l = 0; l < nl; ++l) il.v[l] = 1.0 / slm->wavelengths[l];
    float2 *pixtab = at<float2>(o, L.pixtab);
    CU(launch_pixtab(nl, H, W, dfx, dfy, il, 64, 32, pixtab, s));  // the tiles of k_exact_accum
    CU(cudaMemsetAsync(acc, 0, sizeof(float2) * (size_t)nl * hw, s));
    CU(launch_fill(Tm, (long long)nl * hw, 1.f, s));
    Plan p;
    GS(get_plan(H, W, nl, 0, &p));
    // even grids: the centred modulations around the mask cancel to constants (see k_exact_mask)
    const bool even = ((H | W) & 1) == 0;
    const float sgn0 = ((H / 2 + W / 2) & 1) ? -1.f : 1.f;
    const float uscale = even ? (float)(dfx * dfy) * sgn0 : 1.f;
    const float vscale = even ? (float)(slm->pitch_x * slm->pitch_y) * sgn0 : 1.f;
    timer_mark(o, GWS_TIMER_SPLAT_FWD, 0, s);  // the whole front-to-back loop
    for (long long b0 = 0; b0 < n; b0 += B) {
        const int nb = (int)std::min<long long>(B, n - b0);
        CU(launch_exact_gather(F.sorted, b0, nb, scene, nl, E, 0, s));
        CU(launch_single_spectra(E, nb, nl, H, W, dfx, dfy, il, pixtab, U, s));
        GS(batch_fft(p, H, W, nl, nb, B, U, at<char>(o, L.cufft), CUFFT_INVERSE, s));
        if (!even) CU(launch_modulate(U, 0, nb * nl, H, W, dfx * dfy, 0, s));
        CU(launch_exact_mask(U, Tm, E, nb, nl, hw, o->alpha_min, o->t_binarize, uscale, s));
        // centred forward DFT scaled by px py: the spectrum of each masked field
        if (!even) CU(launch_modulate(U, 0, nb * nl, H, W, 1.0, 1, s));
        GS(batch_fft(p, H, W, nl, nb, B, U, at<char>(o, L.cufft), CUFFT_FORWARD, s));
        if (!even) CU(launch_modulate(U, 0, nb * nl, H, W, slm->pitch_x * slm->pitch_y, 2, s));
        CU(launch_exact_accum(U, acc, pixtab, E, nb, nl, H, W, dfx, dfy, il, even ? 1 : 0, vscale, s));
    }
    timer_mark(o, GWS_TIMER_SPLAT_FWD, 1, s);
    timer_mark(o, GWS_TIMER_FFT, 0, s);
    if (o->domain == GWS_DOMAIN_FIELD) {
        CU(launch_modulate(acc, 0, nl, H, W, 1.0, 3, s));
        GS(exec_fft(p, acc, at<char>(o, L.cufft), 0, CUFFT_INVERSE, s));
        CU(launch_modulate(acc, 0, nl, H, W, dfx * dfy, 0, s));
    }
    timer_mark(o, GWS_TIMER_FFT, 1, s);
    timer_mark(o, GWS_TIMER_TOTAL, 1, s);
    return GWS_OK;
}

// One frame of partially coherent GWS (Eq. 14 summed as Eq. 12): batches of B Gaussians; each
// batch's fields at the origin on their own planes (dense one-Gaussian spectra and a batched
// inverse FFT), times c o kappa, back to the spectrum by a centred forward DFT (scale px py), and
// accumulated with the ramps e^{-j 2 pi f . mu}; a final centred inverse DFT gives the field.
static gws_status pc_forward(const gws_gaussians *scene, long long n, const gws_slm *slm, const gws_opts *o,
                             const Layout &L, const Front &F, void *out, cudaStream_t s) {
    NvtxRange nvtx("gws: partial coherence");
    const int nl = slm->n_lambda, H = slm->H, W = slm->W;
    const long long hw = (long long)H * W;
    const double dfx = 1.0 / (W * slm->pitch_x), dfy = 1.0 / (H * slm->pitch_y);
    const int B = L.ex_B;
    float2 *acc = static_cast<float2 *>(out);
    float2 *U = at<float2>(o, L.ex_U);
    float2 *kappa = at<float2>(o, L.pc_kappa);
    double *ysum = at<double>(o, L.pc_ysum);
    char *arr = at<char>(o, L.ex_arr);
    ExactBatch E;
    E.mean = reinterpret_cast<double *>(arr);
    E.zk = E.mean + 3 * B;
    E.mu = E.zk + B;
    E.quat = reinterpret_cast<float *>(E.mu + 3 * B);
    E.scale = E.quat + 4 * B;
    E.opacity = E.scale + 2 * B;
    E.amp = E.opacity + B;
    E.co = E.amp + (size_t)B * nl;
    E.ok = E.co + (size_t)B * nl;
    E.rr = E.ok + B;
    E.status = at<int>(o, L.status);
    E.n = n;
    InvLam il;
    std::memset(&il, 0, sizeof il);
    for (int l = 0; l < nl; ++l) il.v[l] = 1.0 / slm->wavelengths[l];
    Plan p;
    GS(get_plan(H, W, nl, 0, &p));
    timer_mark(o, GWS_TIMER_SPLAT_FWD, 0, s);  // the kernel patterns and the batch loop
    // each frame's kernel pattern: kappa(x) = sum_f K(f) e^{j 2 pi f . x}, normalised in launch_pc_apply
    const int nf = pc_frames(o);
    const size_t slab = (size_t)nl * hw;
    CU(cudaMemsetAsync(ysum, 0, sizeof(double) * nl * nf, s));
    for (int f = 0; f < nf; ++f) {
        float2 *kf = kappa + (size_t)f * slab;
        CU(launch_pc_kernel(kf, ysum + (size_t)f * nl, o->pc_l, o->pc_m, (unsigned long long)o->pc_seed,
                            (unsigned long long)o->pc_frame + (unsigned long long)f, nl, H, W, dfx, dfy, il, s));
        CU(launch_modulate(kf, 0, nl, H, W, 1.0, 3, s));
        GS(exec_fft(p, kf, at<char>(o, L.cufft), 0, CUFFT_INVERSE, s));
        CU(launch_modulate(kf, 0, nl, H, W, 1.0, 0, s));
    }
    float2 *pixtab = at<float2>(o, L.pixtab);
    CU(launch_pixtab(nl, H, W, dfx, dfy, il, 64, 32, pixtab, s));  // the tiles of the accumulation
    CU(cudaMemsetAsync(acc, 0, sizeof(float2) * slab * nf, s));
    const bool even = ((H | W) & 1) == 0;
    const float sgn0 = ((H / 2 + W / 2) & 1) ? -1.f : 1.f;
    const float uscale = even ? (float)(dfx * dfy) * sgn0 : 1.f;
    const float vscale = even ? (float)(slm->pitch_x * slm->pitch_y) * sgn0 : 1.f;
    // one frame works on the batch's fields in place; several frames share them (computed once per
    // batch) and work on a copy each
    float2 *V = nf > 1 ? at<float2>(o, L.ex_U2) : U;
    for (long long b0 = 0; b0 < n; b0 += B) {
        const int nb = (int)std::min<long long>(B, n - b0);
        CU(launch_exact_gather(F.sorted, b0, nb, scene, nl, E, 1, s));
        CU(launch_single_spectra(E, nb, nl, H, W, dfx, dfy, il, pixtab, U, s));
        GS(batch_fft(p, H, W, nl, nb, B, U, at<char>(o, L.cufft), CUFFT_INVERSE, s));
        if (!even) CU(launch_modulate(U, 0, nb * nl, H, W, dfx * dfy, 0, s));
        for (int f = 0; f < nf; ++f) {
            CU(launch_pc_apply(U, V, kappa + (size_t)f * slab, ysum + (size_t)f * nl, E, nb, nl, hw, uscale, s));
            if (!even) CU(launch_modulate(V, 0, nb * nl, H, W, 1.0, 1, s));
            GS(batch_fft(p, H, W, nl, nb, B, V, at<char>(o, L.cufft), CUFFT_FORWARD, s));
            if (!even) CU(launch_modulate(V, 0, nb * nl, H, W, slm->pitch_x * slm->pitch_y, 2, s));
            CU(launch_pc_accum(V, acc + (size_t)f * slab, pixtab, E, nb, nl, H, W, dfx, dfy, il,
                               o->phase_match ? 1 : 0, even ? 1 : 0, vscale, s));
        }
    }
    timer_mark(o, GWS_TIMER_SPLAT_FWD, 1, s);
    timer_mark(o, GWS_TIMER_FFT, 0, s);
    if (o->domain == GWS_DOMAIN_FIELD) {
        for (int f = 0; f < nf; ++f) {
            float2 *af = acc + (size_t)f * slab;
            CU(launch_modulate(af, 0, nl, H, W, 1.0, 3, s));
            GS(exec_fft(p, af, at<char>(o, L.cufft), 0, CUFFT_INVERSE, s));
            CU(launch_modulate(af, 0, nl, H, W, dfx * dfy, 0, s));
        }
    }
    timer_mark(o, GWS_TIMER_FFT, 1, s);
    timer_mark(o, GWS_TIMER_TOTAL, 1, s);
    return GWS_OK;
}

static gws_status forward_impl(const gws_gaussians *scenes, const int64_t *n, int n_scenes, const gws_slm *slm,
                               const gws_opts *o, void *const *out) {
    GS(check_slm(slm));
    GS(check_opts(o));
    if (n_scenes < 1 || n_scenes > GWS_MAX_SCENES || !n || !out) return GWS_ERR_INVALID_ARG;
    long long n_total = 0;
    for (int k = 0; k < n_scenes; ++k) {
        GS(check_gaussians(&scenes[k], n[k]));
        if (!out[k]) return GWS_ERR_INVALID_ARG;
        n_total += n[k];
    }
    if (n_total > (1ll << 30)) return GWS_ERR_INVALID_ARG;
    const bool fft = o->domain == GWS_DOMAIN_FIELD;
    Layout L;
    GS(plan_layout(n_total, n_scenes, slm, o, &L, fft));
    GS(check_workspace(o, L));
    cudaStream_t s = (cudaStream_t)o->stream;
    CanaryGuard guard(o, L, s);
    NvtxRange nvtx_call("gws_forward");
    timers_reset(o);
    timer_mark(o, GWS_TIMER_TOTAL, 0, s);
    const int nl = slm->n_lambda, H = slm->H, W = slm->W;
    const bool dbl = o->prec == GWS_PREC_FP64;
    const size_t slice = (size_t)H * W * (dbl ? 16 : 8);
    CU(cudaMemsetAsync(at<char>(o, L.status), 0, 16, s));
    if (n_total == 0) {
        // partial coherence writes pc_frames slabs of n_lambda x H x W (one per frame)
        const size_t frames = o->blend == GWS_BLEND_PARTIAL_COHERENT ? (size_t)pc_frames(o) : 1;
        for (int k = 0; k < n_scenes; ++k) CU(cudaMemsetAsync(out[k], 0, slice * nl * frames, s));
        return GWS_OK;
    }
    Front F;
    if (o->blend == GWS_BLEND_EXACT || o->blend == GWS_BLEND_PARTIAL_COHERENT) {
        if (dbl || n_scenes != 1) return GWS_ERR_UNSUPPORTED;
        GS(run_front(scenes, n, n_scenes, slm, o, L, false, &F, s));
        if (o->blend == GWS_BLEND_PARTIAL_COHERENT) return pc_forward(scenes, n_total, slm, o, L, F, out[0], s);
        return exact_forward(scenes, n_total, slm, o, L, F, out[0], s);
    }
    GS(run_front(scenes, n, n_scenes, slm, o, L, o->blend == GWS_BLEND_SORTED_T, &F, s));
    const double dfx = 1.0 / (W * slm->pitch_x), dfy = 1.0 / (H * slm->pitch_y);
    if (dbl) {
        Rec64 *r64 = at<Rec64>(o, L.rec64);
        double *w64 = at<double>(o, L.w64);
        CU(launch_rec64(at<GPre>(o, L.gpre), at<float>(o, L.ampc), F.sorted, F.T_sorted, n_total, nl, r64, w64, s));
        Splat64Args a;
        std::memset(&a, 0, sizeof a);
        a.rec = r64;
        a.w = w64;
        a.segs = F.S;
        a.H = H;
        a.W = W;
        a.dfx = dfx;
        a.dfy = dfy;
        for (int l = 0; l < nl; ++l) a.inv_lam[l] = 1.0 / slm->wavelengths[l];
        a.field_mode = fft ? 1 : 0;
        a.phase_match = o->phase_match ? 1 : 0;
        a.status = at<int>(o, L.status);
        for (int k = 0; k < n_scenes; ++k) a.out[k] = out[k];
        NvtxRange nvtx("gws: splat (FP64)");
        timer_mark(o, GWS_TIMER_SPLAT_FWD, 0, s);
        CU(launch_splat_fp64(a, s));
        timer_mark(o, GWS_TIMER_SPLAT_FWD, 1, s);
    } else {
        Rec *rec = nullptr;
        GS(run_records(F, slm, o, L, 0, s, &rec));
        const int n_seg = n_scenes * nl;
        const TileCfg tc = tile_cfg(L.cfg);
        unsigned long long *ik0 = at<unsigned long long>(o, L.ikey0), *ik1 = at<unsigned long long>(o, L.ikey1);
        unsigned *iv0 = at<unsigned>(o, L.ival0), *iv1 = at<unsigned>(o, L.ival1);
        int *icount = at<int>(o, L.icount);
        CU(launch_items(at<float>(o, L.Rr), F.S, n_seg, H, W, tc.tw, tc.th, L.tiles_x, L.n_tiles, dfx, dfy, ik0, iv0,
                        icount, s));
        const long long n_items = (long long)n_seg * L.n_tiles;
        CU(radix_sort<unsigned long long>(ik0, ik1, iv0, iv1, n_items, 0, 32 + seg_bits(n_seg), at<unsigned>(o, L.hist),
                                          s, at<int>(o, L.status)));
        CU(cudaMemsetAsync(at<int>(o, L.queue), 0, 16, s));
        // per-pixel (f_z - f0_z, log2(1/f_z)) of this configuration's tiles, once per call (FP64)
        InvLam il;
        std::memset(&il, 0, sizeof il);
        for (int l = 0; l < nl; ++l) il.v[l] = 1.0 / slm->wavelengths[l];
        float2 *ftab = at<float2>(o, L.pixtab);
        CU(launch_pixtab(nl, H, W, dfx, dfy, il, tc.tw, tc.th, ftab, s));
        SplatArgs a;
        std::memset(&a, 0, sizeof a);
        a.pixtab = ftab;
        a.rec = rec;
        a.items = iv0;
        a.item_count = icount;
        a.n_items = (int)n_items;
        a.queue = at<int>(o, L.queue);
        a.status = at<int>(o, L.status);
        a.segs = F.S;
        a.H = H;
        a.W = W;
        a.tiles_x = L.tiles_x;
        a.n_tiles = L.n_tiles;
        a.dfx = dfx;
        a.dfy = dfy;
        for (int l = 0; l < nl; ++l) a.inv_lam[l] = 1.0 / slm->wavelengths[l];
        {
            const FootParams FPa = foot_params(slm, o);
            for (int l = 0; l < nl; ++l) a.dzmax[l] = FPa.dzmax[l];
        }
        a.field_mode = fft ? 1 : 0;
        a.phase_match = o->phase_match ? 1 : 0;
        a.timeout = o->timeout_cycles;
        a.debug = o->debug_flags;
        for (int k = 0; k < n_scenes; ++k) a.out[k] = out[k];
        const int grid = (int)std::min<long long>(n_items, (long long)num_sms() * splat_mixed_ctas_per_sm(L.cfg));
        NvtxRange nvtx("gws: splat");
        timer_mark(o, GWS_TIMER_SPLAT_FWD, 0, s);
        CU(launch_splat_mixed(L.cfg, a, grid, s));
        timer_mark(o, GWS_TIMER_SPLAT_FWD, 1, s);
    }
    if (fft) {
        NvtxRange nvtx("gws: inverse DFT");
        Plan p, pb;
        GS(get_plan(H, W, nl, dbl, &p));
        timer_mark(o, GWS_TIMER_FFT, 0, s);
        bool contiguous = n_scenes > 1;
        for (int k = 1; k < n_scenes && contiguous; ++k)
            contiguous = static_cast<char *>(out[k]) == static_cast<char *>(out[0]) + (size_t)k * nl * slice;
        if (contiguous && cached_plan(H, W, n_scenes * nl, dbl, &pb)) {
            GS(exec_fft(pb, out[0], at<char>(o, L.cufft), dbl, CUFFT_INVERSE, s));
            CU(launch_modulate(out[0], dbl, n_scenes * nl, H, W, dfx * dfy, 0, s));
        } else {
            for (int k = 0; k < n_scenes; ++k) {
                GS(exec_fft(p, out[k], at<char>(o, L.cufft), dbl, CUFFT_INVERSE, s));
                CU(launch_modulate(out[k], dbl, nl, H, W, dfx * dfy, 0, s));
            }
        }
        timer_mark(o, GWS_TIMER_FFT, 1, s);
    }
    timer_mark(o, GWS_TIMER_TOTAL, 1, s);
    return GWS_OK;
}

}  // namespace gws

namespace gws {
// the argument checks of the encoding, shared by gws_encode and gws_encode_noalloc
gws_status check_encode_args(const void *field, const gws_slm *slm, const gws_opts *opts, const float *phase_out,
                             float amp_scale) {
    GS(check_slm(slm));
    GS(check_opts(opts));
    if (!field || !phase_out || !std::isfinite(amp_scale)) return GWS_ERR_INVALID_ARG;
    return GWS_OK;
}
}  // namespace gws

using namespace gws;

extern "C" {

void gws_opts_default(gws_opts *o) {
    if (!o) return;
    std::memset(o, 0, sizeof *o);
    o->blend = GWS_BLEND_OIT;
    o->prec = GWS_PREC_MIXED;
    o->domain = GWS_DOMAIN_FIELD;
    o->phase_match = 0;
    o->trunc_eps = 1e-5f;
    o->alpha_min = 1.0f / 255.0f;
    o->tile_cfg = 0;
    o->debug_flags = 0;
    o->timeout_cycles = 2000000000ull;
}

const char *gws_status_string(gws_status s) {
    switch (s) {
        case GWS_OK: return "GWS_OK";
        case GWS_ERR_INVALID_ARG: return "GWS_ERR_INVALID_ARG";
        case GWS_ERR_WORKSPACE: return "GWS_ERR_WORKSPACE";
        case GWS_ERR_CUDA: return "GWS_ERR_CUDA";
        case GWS_ERR_NONFINITE: return "GWS_ERR_NONFINITE";
        case GWS_ERR_TIMEOUT: return "GWS_ERR_TIMEOUT";
        case GWS_ERR_UNSUPPORTED: return "GWS_ERR_UNSUPPORTED";
        case GWS_ERR_BOUNDS: return "GWS_ERR_BOUNDS";
    }
    return "GWS_ERR_UNKNOWN";
}

int gws_version(void) { return GWS_ABI_VERSION; }

int gws_tile_config_ext(int id, int *desc, int n_desc) {
    const int n = n_tile_cfgs();
    if (desc && id >= 1 && id <= n) {
        const TileCfg c = tile_cfg(id);
        const int v[9] = {c.tw, c.th, c.px, c.ru, c.chunk, c.stages, c.ctas, c.npoly, c.step};
        for (int i = 0; i < 9 && i < n_desc; ++i) desc[i] = v[i];
    }
    return n;
}

int gws_tile_config(int id, int *desc) { return gws_tile_config_ext(id, desc, 8); }

int gws_last_launch_count(void) { return t_launches; }

gws_status gws_workspace_size(const int64_t *n, int n_scenes, const gws_slm *slm, const gws_opts *opts,
                              size_t *bytes) {
    if (!bytes || !n || n_scenes < 1 || n_scenes > GWS_MAX_SCENES) return GWS_ERR_INVALID_ARG;
    GS(check_slm(slm));
    GS(check_opts(opts));
    long long tot = 0;
    for (int k = 0; k < n_scenes; ++k) {
        if (n[k] < 0) return GWS_ERR_INVALID_ARG;
        tot += n[k];
    }
    if (tot > (1ll << 30)) return GWS_ERR_INVALID_ARG;
    Layout L;
    GS(plan_layout(tot, n_scenes, slm, opts, &L, opts->domain == GWS_DOMAIN_FIELD));
    *bytes = L.total;
    return GWS_OK;
}

gws_status gws_prepare(const gws_slm *slm, const gws_opts *opts, int n_scenes) {
    GS(check_slm(slm));
    GS(check_opts(opts));
    if (n_scenes < 1 || n_scenes > GWS_MAX_SCENES) return GWS_ERR_INVALID_ARG;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev < 1) return GWS_ERR_CUDA;
    CU(prepare_splat_kernels());
    CU(prepare_bwd_kernels());
    Plan p;
    GS(get_plan(slm->H, slm->W, slm->n_lambda, 0, &p));
    if (n_scenes > 1) GS(get_plan(slm->H, slm->W, n_scenes * slm->n_lambda, opts->prec == GWS_PREC_FP64, &p));
    if (opts->blend == GWS_BLEND_EXACT || opts->blend == GWS_BLEND_PARTIAL_COHERENT) {
        GS(get_plan(slm->H, slm->W, exact_batch(opts) * slm->n_lambda, 0, &p));
    }
    return get_plan(slm->H, slm->W, slm->n_lambda, opts->prec == GWS_PREC_FP64, &p);
}

gws_status gws_forward(const gws_gaussians *g, int64_t n, const gws_slm *slm, const gws_opts *opts, void *field_out) {
    gws_gaussians empty;
    std::memset(&empty, 0, sizeof empty);
    void *outs[1] = {field_out};
    int64_t ns[1] = {n};
    t_launches = 0;
    return forward_impl(g ? g : &empty, ns, 1, slm, opts, outs);
}

gws_status gws_forward_batched(const gws_gaussians *scenes, const int64_t *n, int n_scenes, const gws_slm *slm,
                               const gws_opts *opts, void *const *field_out) {
    if (!scenes) return GWS_ERR_INVALID_ARG;
    if (opts && (opts->blend == GWS_BLEND_EXACT || opts->blend == GWS_BLEND_PARTIAL_COHERENT))
        return GWS_ERR_UNSUPPORTED;
    t_launches = 0;
    return forward_impl(scenes, n, n_scenes, slm, opts, field_out);
}

gws_status gws_encode(const void *field, const gws_slm *slm, const gws_opts *opts, float *phase_out,
                      float amp_scale) {
    t_launches = 0;
    GS(gws::check_encode_args(field, slm, opts, phase_out, amp_scale));
    Layout L;
    GS(plan_layout(0, 1, slm, opts, &L, false));
    if (amp_scale <= 0.f) {
        if (!opts->workspace || (((uintptr_t)opts->workspace) & 255u) || opts->workspace_bytes < L.amax + 8 * GWS_MAX_LAMBDA)
            return GWS_ERR_WORKSPACE;
    }
    cudaStream_t s = (cudaStream_t)opts->stream;
    unsigned long long *amax = opts->workspace ? at<unsigned long long>(opts, L.amax) : nullptr;
    NvtxRange nvtx("gws_encode");
    timers_reset(opts);
    timer_mark(opts, GWS_TIMER_ENCODE, 0, s);
    CU(launch_encode(field, opts->prec == GWS_PREC_FP64, slm->n_lambda, slm->H, slm->W, amax, (double)amp_scale,
                     phase_out, s));
    timer_mark(opts, GWS_TIMER_ENCODE, 1, s);
    return GWS_OK;
}

gws_status gws_get_device_status(const gws_opts *opts) {
    if (!opts || !opts->workspace) return GWS_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)opts->stream;
    int h = 0;
    CU(cudaMemcpyAsync(&h, opts->workspace, sizeof(int), cudaMemcpyDeviceToHost, s));
    CU(cudaStreamSynchronize(s));
    CU(cudaMemsetAsync(opts->workspace, 0, sizeof(int), s));
    if (h & ST_BOUNDS) return GWS_ERR_BOUNDS;
    if (h & ST_NONFINITE) return GWS_ERR_NONFINITE;
    if (h & ST_TIMEOUT) return GWS_ERR_TIMEOUT;
    if (h & ST_BADVALUE) return GWS_ERR_INVALID_ARG;
    return GWS_OK;
}

gws_status gws_depth_order(const gws_gaussians *g, int64_t n, const gws_opts *opts, int32_t *order_out) {
    t_launches = 0;
    GS(check_opts(opts));
    GS(check_gaussians(g, n));
    if (n > 0 && !order_out) return GWS_ERR_INVALID_ARG;
    double lam = 5e-7;
    gws_slm slm{1, 1, 1e-6, 1e-6, 1, &lam};
    Layout L;
    GS(plan_layout(n, 1, &slm, opts, &L, false));
    GS(check_workspace(opts, L));
    CanaryGuard guard(opts, L, (cudaStream_t)opts->stream);
    if (n == 0) return GWS_OK;
    cudaStream_t s = (cudaStream_t)opts->stream;
    CU(cudaMemsetAsync(at<char>(opts, L.status), 0, 16, s));
    Front F;
    int64_t ns[1] = {n};
    // amplitudes are read with n_lambda = 1: only amp[i][0] is touched
    GS(run_front(g, ns, 1, &slm, opts, L, false, &F, s));
    CU(cudaMemcpyAsync(order_out, F.sorted, sizeof(int32_t) * n, cudaMemcpyDeviceToDevice, s));
    return GWS_OK;
}

gws_status gws_transmittance(const gws_gaussians *g, int64_t n, const gws_opts *opts, double *T_out) {
    t_launches = 0;
    GS(check_opts(opts));
    GS(check_gaussians(g, n));
    if (n > 0 && !T_out) return GWS_ERR_INVALID_ARG;
    double lam = 5e-7;
    gws_slm slm{1, 1, 1e-6, 1e-6, 1, &lam};
    Layout L;
    GS(plan_layout(n, 1, &slm, opts, &L, false));
    GS(check_workspace(opts, L));
    CanaryGuard guard(opts, L, (cudaStream_t)opts->stream);
    if (n == 0) return GWS_OK;
    cudaStream_t s = (cudaStream_t)opts->stream;
    CU(cudaMemsetAsync(at<char>(opts, L.status), 0, 16, s));
    Front F;
    int64_t ns[1] = {n};
    GS(run_front(g, ns, 1, &slm, opts, L, true, &F, s));
    CU(cudaMemcpyAsync(T_out, F.T_g, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
    return GWS_OK;
}

gws_status gws_footprints(const gws_gaussians *g, int64_t n, const gws_slm *slm, const gws_opts *opts, int l,
                          float *ellipse_out) {
    t_launches = 0;
    GS(check_slm(slm));
    GS(check_opts(opts));
    GS(check_gaussians(g, n));
    if (l < 0 || l >= slm->n_lambda || (n > 0 && !ellipse_out)) return GWS_ERR_INVALID_ARG;
    Layout L;
    GS(plan_layout(n, 1, slm, opts, &L, false));
    GS(check_workspace(opts, L));
    CanaryGuard guard(opts, L, (cudaStream_t)opts->stream);
    if (n == 0) return GWS_OK;
    cudaStream_t s = (cudaStream_t)opts->stream;
    CU(cudaMemsetAsync(at<char>(opts, L.status), 0, 16, s));
    SceneTable T;
    std::memset(&T, 0, sizeof T);
    T.n_scenes = 1;
    T.n_lambda = slm->n_lambda;
    T.off[1] = n;
    T.mean[0] = g->mean;
    T.quat[0] = g->quat;
    T.scale[0] = g->scale;
    T.opacity[0] = g->opacity;
    T.amp[0] = g->amp;
    GPre *gp = at<GPre>(opts, L.gpre);
    CU(launch_prep(T, n, gp, at<float>(opts, L.ampc), at<unsigned long long>(opts, L.dkey0),
                   at<unsigned>(opts, L.dval0), at<int>(opts, L.status), s));
    const FootParams FP = foot_params(slm, opts);
    CU(launch_foot_inspect(gp, n, FP.rho, FP.dzmax[l], ellipse_out, s));
    return GWS_OK;
}

float gws_kernel_time_ms(int which) {
    if (which < 0 || which > 4 || !t_timers.made || !t_timers.used[which]) return -1.f;
    if (cudaEventSynchronize(t_timers.ev[which][1]) != cudaSuccess) return -1.f;
    float ms = -1.f;
    if (cudaEventElapsedTime(&ms, t_timers.ev[which][0], t_timers.ev[which][1]) != cudaSuccess) return -1.f;
    return ms;
}

gws_status gws_footprint_pairs(const gws_gaussians *g, int64_t n, const gws_slm *slm, const gws_opts *opts,
                               unsigned long long *pairs) {
    t_launches = 0;
    GS(check_slm(slm));
    GS(check_opts(opts));
    GS(check_gaussians(g, n));
    if (!pairs) return GWS_ERR_INVALID_ARG;
    *pairs = 0;
    Layout L;
    GS(plan_layout(n, 1, slm, opts, &L, false));
    GS(check_workspace(opts, L));
    CanaryGuard guard(opts, L, (cudaStream_t)opts->stream);
    if (n == 0) return GWS_OK;
    cudaStream_t s = (cudaStream_t)opts->stream;
    CU(cudaMemsetAsync(at<char>(opts, L.status), 0, 16, s));
    SceneTable T;
    std::memset(&T, 0, sizeof T);
    T.n_scenes = 1;
    T.n_lambda = slm->n_lambda;
    T.off[1] = n;
    T.mean[0] = g->mean;
    T.quat[0] = g->quat;
    T.scale[0] = g->scale;
    T.opacity[0] = g->opacity;
    T.amp[0] = g->amp;
    GPre *gp = at<GPre>(opts, L.gpre);
    CU(launch_prep(T, n, gp, at<float>(opts, L.ampc), at<unsigned long long>(opts, L.dkey0),
                   at<unsigned>(opts, L.dval0), at<int>(opts, L.status), s));
    const FootParams FP = foot_params(slm, opts);
    unsigned long long *acc = at<unsigned long long>(opts, L.queue);
    CU(cudaMemsetAsync(acc, 0, 8, s));
    CU(launch_count_pairs(gp, n, slm->n_lambda, FP, slm->H, slm->W, 1.0 / (slm->W * slm->pitch_x),
                          1.0 / (slm->H * slm->pitch_y), acc, s));
    CU(cudaMemcpyAsync(pairs, acc, 8, cudaMemcpyDeviceToHost, s));
    CU(cudaStreamSynchronize(s));
    return GWS_OK;
}

gws_status gws_backward(const gws_gaussians *g, int64_t n, const gws_slm *slm, const gws_opts *opts,
                        const void *grad_field, gws_gaussians_grad *out) {
    t_launches = 0;
    GS(check_slm(slm));
    GS(check_opts(opts));
    GS(check_gaussians(g, n));
    if (!grad_field || !out) return GWS_ERR_INVALID_ARG;
    if (n > 0 && (!out->mean || !out->quat || !out->scale || !out->opacity || !out->amp)) return GWS_ERR_INVALID_ARG;
    if (opts->prec != GWS_PREC_MIXED) return GWS_ERR_UNSUPPORTED;
    // the exact blend and partial coherence are forward-only
    if (opts->blend == GWS_BLEND_EXACT || opts->blend == GWS_BLEND_PARTIAL_COHERENT) return GWS_ERR_UNSUPPORTED;
    const bool sorted_t = opts->blend == GWS_BLEND_SORTED_T;
    const bool fft = opts->domain == GWS_DOMAIN_FIELD;
    Layout L;
    GS(plan_layout(n, 1, slm, opts, &L, fft));
    GS(check_workspace(opts, L));
    CanaryGuard guard(opts, L, (cudaStream_t)opts->stream);
    cudaStream_t s = (cudaStream_t)opts->stream;
    NvtxRange nvtx_call("gws_backward");
    timers_reset(opts);
    timer_mark(opts, GWS_TIMER_TOTAL, 0, s);
    CU(cudaMemsetAsync(at<char>(opts, L.status), 0, 16, s));
    if (n == 0) return GWS_OK;
    const int nl = slm->n_lambda, H = slm->H, W = slm->W;
    const double dfx = 1.0 / (W * slm->pitch_x), dfy = 1.0 / (H * slm->pitch_y);
    Front F;
    int64_t ns[1] = {n};
    GS(run_front(g, ns, 1, slm, opts, L, opts->blend == GWS_BLEND_SORTED_T, &F, s));
    Rec *rec = nullptr;
    GS(run_records(F, slm, opts, L, 1, s, &rec));
    // dL/du_SLM: the adjoint of the centred inverse DFT (dfx dfy x centred forward DFT)
    const float2 *gsrc = static_cast<const float2 *>(grad_field);
    if (fft) {
        NvtxRange nvtx("gws: adjoint DFT");
        float2 *gs = at<float2>(opts, L.gspec);
        CU(cudaMemcpyAsync(gs, grad_field, sizeof(float2) * (size_t)nl * H * W, cudaMemcpyDeviceToDevice, s));
        CU(launch_modulate(gs, 0, nl, H, W, 1.0, 1, s));
        Plan p;
        GS(get_plan(H, W, nl, 0, &p));
        timer_mark(opts, GWS_TIMER_FFT, 0, s);
        GS(exec_fft(p, gs, at<char>(opts, L.cufft), 0, CUFFT_FORWARD, s));
        timer_mark(opts, GWS_TIMER_FFT, 1, s);
        CU(launch_modulate(gs, 0, nl, H, W, dfx * dfy, 2, s));
        gsrc = gs;
    }
    InvLam il;
    std::memset(&il, 0, sizeof il);
    for (int l = 0; l < nl; ++l) il.v[l] = 1.0 / slm->wavelengths[l];
    float4 *btab = at<float4>(opts, L.gtiles);
    float2 *bps = at<float2>(opts, L.pixtab);
    CU(launch_bwd_tables(nl, H, W, dfx, dfy, il, gsrc, btab, bps, s));
    CU(cudaMemsetAsync(at<int>(opts, L.queue), 0, 16, s));
    BwdArgs a;
    std::memset(&a, 0, sizeof a);
    a.rec = rec;
    a.tab = btab;
    a.ps = bps;
    a.acc = at<double>(opts, L.bacc);
    a.queue = at<int>(opts, L.queue);
    a.status = at<int>(opts, L.status);
    a.segs = F.S;
    a.H = H;
    a.W = W;
    a.tiles_x = bwd_tiles_x(W);
    a.tiles_y = bwd_tiles_y(H);
    a.dfx = dfx;
    a.dfy = dfy;
    for (int l = 0; l < nl; ++l) a.inv_lam[l] = il.v[l];
    {
        const FootParams FPa = foot_params(slm, opts);
        for (int l = 0; l < nl; ++l) a.dzmax[l] = FPa.dzmax[l];
    }
    a.phase_match = opts->phase_match ? 1 : 0;
    const int B = bwd_block_size();
    a.n_items = (int)(nl * ((n + B - 1) / B));
    const int grid = (int)std::min<long long>(a.n_items, (long long)num_sms() * bwd_ctas_per_sm());
    {
        NvtxRange nvtx("gws: splat backward");
        timer_mark(opts, GWS_TIMER_SPLAT_BWD, 0, s);
        CU(launch_splat_bwd(a, grid, s));
        timer_mark(opts, GWS_TIMER_SPLAT_BWD, 1, s);
    }
    GradArgs G;
    std::memset(&G, 0, sizeof G);
    G.mean = out->mean;
    G.quat = out->quat;
    G.scale = out->scale;
    G.opacity = out->opacity;
    G.amp = out->amp;
    G.dT = sorted_t ? at<double>(opts, L.dT) : nullptr;
    G.phase_match = opts->phase_match ? 1 : 0;
    G.status = at<int>(opts, L.status);
    for (int l = 0; l < nl; ++l) G.inv_lam[l] = il.v[l];
    CU(launch_grad_assemble(at<GPre>(opts, L.gpre), at<float>(opts, L.ampc), F.T_g, at<int>(opts, L.invrec),
                            at<double>(opts, L.bacc), g->quat, n, nl, G, s));
    if (sorted_t)  // cross terms through T_i (Eq. 5-6 reading): on the query's mean and on every front Gaussian
        CU(launch_tgrad(at<TData>(opts, L.tdata), at<TQuery>(opts, L.tq), at<GPre>(opts, L.gpre), F.sorted,
                        at<double>(opts, L.dT), g->quat, F.S, n, (double)opts->alpha_min, out->mean, out->quat,
                        out->scale, out->opacity, s));
    timer_mark(opts, GWS_TIMER_TOTAL, 1, s);
    return GWS_OK;
}

gws_status gws_tune_get(const gws_slm *slm, int *cfg) {
    if (!cfg) return GWS_ERR_INVALID_ARG;
    GS(check_slm(slm));
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tuned.find(std::make_tuple(slm->H, slm->W, slm->n_lambda));
    *cfg = it != g_tuned.end() ? it->second : 0;
    return GWS_OK;
}

gws_status gws_tune_set(const gws_slm *slm, int cfg) {
    GS(check_slm(slm));
    if (cfg < 0 || cfg > n_tile_cfgs()) return GWS_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(g_tune_mu);
    const auto key = std::make_tuple(slm->H, slm->W, slm->n_lambda);
    if (cfg == 0) g_tuned.erase(key);
    else g_tuned[key] = cfg;
    return GWS_OK;
}

gws_status gws_autotune(const gws_gaussians *g, int64_t n, const gws_slm *slm, const gws_opts *opts,
                        void *field_scratch, int *best_cfg) {
    if (!best_cfg || !field_scratch) return GWS_ERR_INVALID_ARG;
    GS(check_slm(slm));
    GS(check_opts(opts));
    GS(check_gaussians(g, n));
    if (opts->prec != GWS_PREC_MIXED || n == 0) {
        *best_cfg = 1;
        return GWS_OK;
    }
    cudaStream_t s = (cudaStream_t)opts->stream;
    float best_ms = 3.0e38f;
    int best = 1;
    for (int c = 1; c <= n_tile_cfgs(); ++c) {
        gws_opts o = *opts;
        o.tile_cfg = c;
        o.domain = GWS_DOMAIN_SPECTRUM;
        o.debug_flags = GWS_DEBUG_TIME_KERNELS;
        float ms = 3.0e38f;
        for (int rep = 0; rep < 2; ++rep) {  // the first run warms caches and the instruction cache
            GS(gws_forward(g, n, slm, &o, field_scratch));
            const float t = gws_kernel_time_ms(GWS_TIMER_SPLAT_FWD);
            if (t < 0) return GWS_ERR_CUDA;
            ms = t;
        }
        if (ms < best_ms) {
            best_ms = ms;
            best = c;
        }
    }
    CU(cudaStreamSynchronize(s));
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        g_tuned[std::make_tuple(slm->H, slm->W, slm->n_lambda)] = best;
    }
    *best_cfg = best;
    return GWS_OK;
}

// ---- triangle primitive ----------------------------------------------------------------------

struct TriLayout {
#ifdef GWS_CHECK_BOUNDS
    size_t canary[kMaxCanaries];
    int n_canary;
#endif
    size_t status, rec, w, cufft, total;
};

static gws_status tri_layout(int64_t n, const gws_slm *slm, bool fft, TriLayout *L) {
    Planner P;
    L->status = P.take(16);  // first: gws_get_device_status reads the word at the workspace start
    L->rec = P.take(sizeof(TriRec) * (size_t)n);
    L->w = P.take(sizeof(float) * (size_t)n * slm->n_lambda);
    size_t work = 0;
    if (fft) {
        Plan p;
        GS(get_plan(slm->H, slm->W, slm->n_lambda, 0, &p));
        work = p.work;
    }
    L->cufft = P.take(std::max<size_t>(work, 16));
    L->total = P.cur;
#ifdef GWS_CHECK_BOUNDS
    L->n_canary = P.n_canary;
    for (int i = 0; i < P.n_canary; ++i) L->canary[i] = P.canary[i];
#endif
    return GWS_OK;
}

gws_status gws_triangles_workspace_size(int64_t n, const gws_slm *slm, const gws_opts *opts, size_t *bytes) {
    GS(check_slm(slm));
    GS(check_opts(opts));
    if (!bytes || n < 0 || n > (1ll << 30)) return GWS_ERR_INVALID_ARG;
    if (opts->prec != GWS_PREC_MIXED) return GWS_ERR_UNSUPPORTED;
    TriLayout L;
    GS(tri_layout(n, slm, opts->domain == GWS_DOMAIN_FIELD, &L));
    *bytes = L.total;
    return GWS_OK;
}

gws_status gws_forward_triangles(const gws_triangles *t, int64_t n, const gws_slm *slm, const gws_opts *opts,
                                 void *field_out) {
    t_launches = 0;
    GS(check_slm(slm));
    GS(check_opts(opts));
    if (!field_out || n < 0 || n > (1ll << 30)) return GWS_ERR_INVALID_ARG;
    if (n > 0 && (!t || !t->vertices || !t->opacity || !t->amp)) return GWS_ERR_INVALID_ARG;
    if (opts->prec != GWS_PREC_MIXED) return GWS_ERR_UNSUPPORTED;
    const bool fft = opts->domain == GWS_DOMAIN_FIELD;
    TriLayout L;
    GS(tri_layout(n, slm, fft, &L));
    if (!opts->workspace || opts->workspace_bytes < L.total) return GWS_ERR_WORKSPACE;
    if (reinterpret_cast<uintptr_t>(opts->workspace) % 256 != 0) return GWS_ERR_WORKSPACE;
    cudaStream_t s = (cudaStream_t)opts->stream;
    CanaryGuard guard(opts, L, s);
    const int nl = slm->n_lambda, H = slm->H, W = slm->W;
    const double dfx = 1.0 / (W * slm->pitch_x), dfy = 1.0 / (H * slm->pitch_y);
    timers_reset(opts);
    timer_mark(opts, GWS_TIMER_TOTAL, 0, s);
    CU(cudaMemsetAsync(at<char>(opts, L.status), 0, 16, s));
    InvLam il;
    std::memset(&il, 0, sizeof il);
    for (int l = 0; l < nl; ++l) il.v[l] = 1.0 / slm->wavelengths[l];
    TriRec *rec = at<TriRec>(opts, L.rec);
    float *w = at<float>(opts, L.w);
    CU(launch_tri_prep(n > 0 ? t->vertices : nullptr, n > 0 ? t->opacity : nullptr, n > 0 ? t->amp : nullptr, n, nl,
                       rec, w, at<int>(opts, L.status), s));
    timer_mark(opts, GWS_TIMER_SPLAT_FWD, 0, s);
    CU(launch_splat_tri(rec, w, n, nl, H, W, dfx, dfy, il, fft ? 1 : 0, opts->phase_match ? 1 : 0,
                        static_cast<float2 *>(field_out), s));
    timer_mark(opts, GWS_TIMER_SPLAT_FWD, 1, s);
    if (fft) {
        Plan p;
        GS(get_plan(H, W, nl, 0, &p));
        timer_mark(opts, GWS_TIMER_FFT, 0, s);
        GS(exec_fft(p, field_out, at<char>(opts, L.cufft), 0, CUFFT_INVERSE, s));
        CU(launch_modulate(field_out, 0, nl, H, W, dfx * dfy, 0, s));
        timer_mark(opts, GWS_TIMER_FFT, 1, s);
    }
    timer_mark(opts, GWS_TIMER_TOTAL, 1, s);
    return GWS_OK;
}

}  // extern "C"
