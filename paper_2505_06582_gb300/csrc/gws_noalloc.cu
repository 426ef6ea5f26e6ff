// gws_noalloc.cu -- double-phase encoding for callers that cannot allocate device memory.
//
// gws_encode needs a few bytes of scratch (the per-wavelength maximum amplitude) from the
// caller's workspace.  Some callers cannot provide one: code hosted inside another
// application that owns every device allocation, or a real-time display loop that fixes
// its memory at start-up and must not call cudaMalloc (which can synchronise the device)
// while frames are in flight.  gws_encode_noalloc gives them the same encoding with that
// scratch in a fixed array inside this library instead.
#include <mutex>

#include "gws_prep.h"

namespace {

constexpr int kMaxDevices = 64;

// One slot per wavelength: the running max of |u|^2 (float or double bits).  Every GPU that
// loads the library holds this array until the process exits.
static __device__ __align__(256) unsigned long long g_encode_scratch[GWS_NOALLOC_MAX_LAMBDA];

std::mutex g_mu;
void *g_scratch_ptr[kMaxDevices] = {nullptr};

// Device address of g_encode_scratch on the current device (host code cannot use the
// symbol itself: on the host it names a stand-in, not device memory).  Looked up once per
// device, with that device current.
cudaError_t scratch_for_current_device(void **out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_scratch_ptr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_encode_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_ptr[dev] = p;
    }
    *out = g_scratch_ptr[dev];
    return cudaSuccess;
}

}  // namespace

extern "C" gws_status gws_encode_noalloc(const void *field, const gws_slm *slm, const gws_opts *opts,
                                         float *phase_out, float amp_scale) {
    if (!slm || !opts || !field || !phase_out) return GWS_ERR_INVALID_ARG;
    if (slm->n_lambda < 1 || slm->n_lambda > GWS_NOALLOC_MAX_LAMBDA) return GWS_ERR_INVALID_ARG;
    if (slm->H < 1 || slm->W < 1 || (long long)slm->H * slm->W > (1ll << 31)) return GWS_ERR_INVALID_ARG;
    if (opts->prec != GWS_PREC_FP64 && opts->prec != GWS_PREC_MIXED) return GWS_ERR_INVALID_ARG;
    if (!(amp_scale == amp_scale) || amp_scale > 3.0e38f) return GWS_ERR_INVALID_ARG;
    void *scratch = nullptr;
    if (scratch_for_current_device(&scratch) != cudaSuccess) return GWS_ERR_CUDA;
    // launch_encode clears the slots it uses before the max reduction (cudaMemsetAsync)
    cudaError_t e = gws::launch_encode(field, opts->prec == GWS_PREC_FP64, slm->n_lambda, slm->H, slm->W,
                                       static_cast<unsigned long long *>(scratch), (double)amp_scale, phase_out,
                                       (cudaStream_t)opts->stream);
    return e == cudaSuccess ? GWS_OK : GWS_ERR_CUDA;
}
