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
// symbol itself: on the host it names a stand-in, not device memory).  Looked up with that
// device current on every call made outside a stream capture (so a context rebuilt after
// cudaDeviceReset gets its new address) and remembered per device; a call made while the
// stream is being captured uses the remembered address, so the first call on a device must
// come before any capture.
cudaError_t scratch_for_current_device(cudaStream_t stream, void **out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    e = cudaStreamIsCapturing(stream, &cap);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lk(g_mu);
    if (cap == cudaStreamCaptureStatusNone) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_encode_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_ptr[dev] = p;
    } else if (!g_scratch_ptr[dev]) {
        return cudaErrorStreamCaptureUnsupported;  // no address yet: the first call came under capture
    }
    *out = g_scratch_ptr[dev];
    return cudaSuccess;
}

}  // namespace

extern "C" gws_status gws_encode_noalloc(const void *field, const gws_slm *slm, const gws_opts *opts,
                                         float *phase_out, float amp_scale) {
    // the same checks as gws_encode, then the limit of the fixed scratch
    const gws_status st = gws::check_encode_args(field, slm, opts, phase_out, amp_scale);
    if (st != GWS_OK) return st;
    if (slm->n_lambda > GWS_NOALLOC_MAX_LAMBDA) return GWS_ERR_INVALID_ARG;
    void *scratch = nullptr;
    if (scratch_for_current_device((cudaStream_t)opts->stream, &scratch) != cudaSuccess) return GWS_ERR_CUDA;
    // launch_encode clears the slots it uses before the max reduction (cudaMemsetAsync)
    cudaError_t e = gws::launch_encode(field, opts->prec == GWS_PREC_FP64, slm->n_lambda, slm->H, slm->W,
                                       static_cast<unsigned long long *>(scratch), (double)amp_scale, phase_out,
                                       (cudaStream_t)opts->stream);
    return e == cudaSuccess ? GWS_OK : GWS_ERR_CUDA;
}
