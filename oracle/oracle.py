"""ctypes wrapper around the FP64 oracle (``gws_oracle.c``).

TEST INFRASTRUCTURE ONLY (tests, smoke check, CPU baseline of the benchmark).
Every function takes numpy arrays and returns numpy arrays in FP64 / complex128.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gws_oracle.c")
_LIB_PATH = os.path.join(_HERE, "_build", "libgws_oracle.so")
_lib = None

BLEND_OIT, BLEND_SORTED_T = 0, 1
ALPHA_MIN = 1.0 / 255.0


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (OpenMP, no FMA contraction, no host-specific flags)."""
    os.makedirs(os.path.dirname(_LIB_PATH), exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fopenmp", "-ffp-contract=off", "-fPIC", "-shared",
                               _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    if _lib is None:
        _lib = C.CDLL(build())
        _lib.gwso_num_threads.restype = C.c_int
    return _lib


def _d(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _p(a):
    return a.ctypes.data_as(C.c_void_p)


def _scene_arrays(scene):
    return (_d(scene.mean), _d(scene.quat), _d(scene.scale), _d(scene.opacity), _d(scene.amp))


def num_threads() -> int:
    return lib().gwso_num_threads()


def set_num_threads(k: int) -> None:
    lib().gwso_set_num_threads(C.c_int(k))


def depth_order(mean) -> np.ndarray:
    mean = _d(mean)
    n = mean.shape[0]
    out = np.empty(n, dtype=np.int64)
    lib().gwso_depth_order(C.c_int64(n), _p(mean), _p(out))
    return out


def transmittance(scene, alpha_min=ALPHA_MIN) -> np.ndarray:
    mean, quat, scale, opa, _ = _scene_arrays(scene)
    T = np.empty(mean.shape[0])
    lib().gwso_transmittance(C.c_int64(mean.shape[0]), _p(mean), _p(quat), _p(scale), _p(opa),
                             C.c_double(alpha_min), _p(T))
    return T


def transmittance_at(scene, which, alpha_min=ALPHA_MIN) -> np.ndarray:
    mean, quat, scale, opa, _ = _scene_arrays(scene)
    which = np.ascontiguousarray(which, dtype=np.int64)
    T = np.empty(which.shape[0])
    lib().gwso_transmittance_at(C.c_int64(mean.shape[0]), _p(mean), _p(quat), _p(scale), _p(opa),
                                C.c_double(alpha_min), C.c_int64(which.shape[0]), _p(which), _p(T))
    return T


def spectrum(scene, slm, blend=BLEND_OIT, phase_match=False, alpha_min=ALPHA_MIN) -> np.ndarray:
    """u_SLM(f), complex128 [n_lambda][H][W]."""
    mean, quat, scale, opa, amp = _scene_arrays(scene)
    wl = _d(slm.wavelengths)
    out = np.empty((slm.n_lambda, slm.H, slm.W, 2))
    lib().gwso_spectrum(C.c_int64(mean.shape[0]), _p(mean), _p(quat), _p(scale), _p(opa), _p(amp),
                        C.c_int(slm.n_lambda), _p(wl), C.c_int(slm.H), C.c_int(slm.W),
                        C.c_double(slm.pitch_x), C.c_double(slm.pitch_y), C.c_int(blend),
                        C.c_int(int(phase_match)), C.c_double(alpha_min), _p(out))
    return out[..., 0] + 1j * out[..., 1]


def spectrum_at(scene, slm, lam_idx, rows, cols, T=None, phase_match=False) -> np.ndarray:
    """u_SLM at samples (lambda index, row, column); T: per-Gaussian transmittance or None."""
    mean, quat, scale, opa, amp = _scene_arrays(scene)
    wl = _d(slm.wavelengths)
    li = np.ascontiguousarray(lam_idx, dtype=np.int32)
    ri = np.ascontiguousarray(rows, dtype=np.int32)
    ci = np.ascontiguousarray(cols, dtype=np.int32)
    Tp = None if T is None else _d(T)
    out = np.empty((li.shape[0], 2))
    lib().gwso_spectrum_at(C.c_int64(mean.shape[0]), _p(mean), _p(quat), _p(scale), _p(opa), _p(amp),
                           None if Tp is None else _p(Tp), C.c_int(slm.n_lambda), _p(wl), C.c_int(slm.H),
                           C.c_int(slm.W), C.c_double(slm.pitch_x), C.c_double(slm.pitch_y),
                           C.c_int(int(phase_match)), C.c_int64(li.shape[0]), _p(li), _p(ri), _p(ci), _p(out))
    return out[:, 0] + 1j * out[:, 1]


def single_terms(mean3, quat4, scale2, lam, H, W, px, py, phase_match=False):
    """(unweighted spectrum [H][W] complex, Gaussian exponent E [H][W]) of one Gaussian."""
    m, q, s = _d(mean3), _d(quat4), _d(scale2)
    term = np.empty((H, W, 2))
    E = np.empty((H, W))
    lib().gwso_single_terms(_p(m), _p(q), _p(s), C.c_double(lam), C.c_int(H), C.c_int(W), C.c_double(px),
                            C.c_double(py), C.c_int(int(phase_match)), _p(term), _p(E))
    return term[..., 0] + 1j * term[..., 1], E


def _cplx(a):
    a = np.ascontiguousarray(a, dtype=np.complex128)
    return a


def idft(spec, px, py) -> np.ndarray:
    """Centred inverse DFT scaled by dfx dfy; spec complex [..., H, W]."""
    spec = _cplx(spec)
    shp = spec.shape
    H, W = shp[-2], shp[-1]
    n = int(np.prod(shp[:-2])) if len(shp) > 2 else 1
    out = np.empty(shp, dtype=np.complex128)
    lib().gwso_idft(C.c_int(n), C.c_int(H), C.c_int(W), C.c_double(px), C.c_double(py), _p(spec), _p(out))
    return out


def idft_adjoint(field_grad, px, py) -> np.ndarray:
    g = _cplx(field_grad)
    shp = g.shape
    H, W = shp[-2], shp[-1]
    n = int(np.prod(shp[:-2])) if len(shp) > 2 else 1
    out = np.empty(shp, dtype=np.complex128)
    lib().gwso_idft_adjoint(C.c_int(n), C.c_int(H), C.c_int(W), C.c_double(px), C.c_double(py), _p(g), _p(out))
    return out


def idft_at(spec2d, px, py, rows, cols) -> np.ndarray:
    spec2d = _cplx(spec2d)
    H, W = spec2d.shape
    ri = np.ascontiguousarray(rows, dtype=np.int32)
    ci = np.ascontiguousarray(cols, dtype=np.int32)
    out = np.empty((ri.shape[0], 2))
    lib().gwso_idft_at(C.c_int(H), C.c_int(W), C.c_double(px), C.c_double(py), _p(spec2d),
                       C.c_int64(ri.shape[0]), _p(ri), _p(ci), _p(out))
    return out[:, 0] + 1j * out[:, 1]


def field(scene, slm, blend=BLEND_OIT, phase_match=False, alpha_min=ALPHA_MIN) -> np.ndarray:
    return idft(spectrum(scene, slm, blend, phase_match, alpha_min), slm.pitch_x, slm.pitch_y)


def encode(field_arr, amp_scale=0.0) -> np.ndarray:
    """Double-phase encoding; field complex [n_lambda][H][W] -> phase float64."""
    f = _cplx(field_arr)
    if f.ndim == 2:
        f = f[None]
    L, H, W = f.shape
    out = np.empty((L, H, W))
    lib().gwso_encode(C.c_int(L), C.c_int(H), C.c_int(W), _p(f), C.c_double(amp_scale), _p(out))
    return out


def backward_spectrum(scene, slm, gspec, blend=BLEND_OIT, phase_match=False, alpha_min=ALPHA_MIN):
    """Analytic gradients given dL/d(spectrum) (PyTorch convention). Returns a dict."""
    mean, quat, scale, opa, amp = _scene_arrays(scene)
    n = mean.shape[0]
    wl = _d(slm.wavelengths)
    g = _cplx(gspec)
    out = dict(mean=np.zeros((n, 3)), quat=np.zeros((n, 4)), scale=np.zeros((n, 2)), opacity=np.zeros(n),
               amp=np.zeros((n, slm.n_lambda)))
    lib().gwso_backward_spectrum(C.c_int64(n), _p(mean), _p(quat), _p(scale), _p(opa), _p(amp),
                                 C.c_int(slm.n_lambda), _p(wl), C.c_int(slm.H), C.c_int(slm.W),
                                 C.c_double(slm.pitch_x), C.c_double(slm.pitch_y), C.c_int(blend),
                                 C.c_int(int(phase_match)), C.c_double(alpha_min), _p(g), _p(out["mean"]),
                                 _p(out["quat"]), _p(out["scale"]), _p(out["opacity"]), _p(out["amp"]))
    return out


def backward_field(scene, slm, gfield, blend=BLEND_OIT, phase_match=False, alpha_min=ALPHA_MIN):
    """Gradients given dL/d(field): the adjoint DFT, then ``backward_spectrum``."""
    return backward_spectrum(scene, slm, idft_adjoint(gfield, slm.pitch_x, slm.pitch_y), blend, phase_match,
                             alpha_min)


def backward_spectrum_at(scene, slm, gspec, which, phase_match=False):
    """Order-invariant gradients of the Gaussians in `which` only (per entry of `which`)."""
    mean, quat, scale, opa, amp = _scene_arrays(scene)
    n = mean.shape[0]
    wl = _d(slm.wavelengths)
    g = _cplx(gspec)
    which = np.ascontiguousarray(which, dtype=np.int64)
    k = which.shape[0]
    out = dict(mean=np.zeros((k, 3)), quat=np.zeros((k, 4)), scale=np.zeros((k, 2)), opacity=np.zeros(k),
               amp=np.zeros((k, slm.n_lambda)))
    lib().gwso_backward_spectrum_at(C.c_int64(n), _p(mean), _p(quat), _p(scale), _p(opa), _p(amp),
                                    C.c_int(slm.n_lambda), _p(wl), C.c_int(slm.H), C.c_int(slm.W),
                                    C.c_double(slm.pitch_x), C.c_double(slm.pitch_y), C.c_int(int(phase_match)),
                                    _p(g), C.c_int64(k), _p(which), _p(out["mean"]), _p(out["quat"]),
                                    _p(out["scale"]), _p(out["opacity"]), _p(out["amp"]))
    return out


def exact_awb(scene, slm, t_eps=ALPHA_MIN, binarize=0.0, with_T=False):
    """Exact alpha wave blending (Algorithm S2): SLM spectrum [n_lambda][H][W] (and T map)."""
    mean, quat, scale, opa, amp = _scene_arrays(scene)
    wl = _d(slm.wavelengths)
    out = np.empty((slm.n_lambda, slm.H, slm.W, 2))
    T = np.empty((slm.n_lambda, slm.H, slm.W)) if with_T else None
    lib().gwso_exact_awb(C.c_int64(mean.shape[0]), _p(mean), _p(quat), _p(scale), _p(opa), _p(amp),
                         C.c_int(slm.n_lambda), _p(wl), C.c_int(slm.H), C.c_int(slm.W), C.c_double(slm.pitch_x),
                         C.c_double(slm.pitch_y), C.c_double(t_eps), C.c_double(binarize), _p(out),
                         None if T is None else _p(T))
    spec = out[..., 0] + 1j * out[..., 1]
    return (spec, T) if with_T else spec
