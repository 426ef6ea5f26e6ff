"""Python binding of libgws (include/gws.h): argument marshalling only.

Every step of the hot path runs in the CUDA library; this module only passes device
pointers, sizes and the current CUDA stream across the C ABI, allocates the caller-side
workspace with PyTorch, and wraps forward / backward in a ``torch.autograd.Function``.
There is no fallback: if ``libgws.so`` is missing or fails to load, every call raises.
"""
from __future__ import annotations

import contextlib
import ctypes as C
import json
import math
import os
import tempfile
import threading
from dataclasses import dataclass

import numpy as np
import torch

from . import _build

BLEND_OIT, BLEND_SORTED_T, BLEND_EXACT, BLEND_PARTIAL_COHERENT = 0, 1, 2, 3
PREC_FP64, PREC_MIXED = 0, 1
DOMAIN_FIELD, DOMAIN_SPECTRUM = 0, 1
PROJ_PERSPECTIVE, PROJ_ORTHOGRAPHIC = 0, 1
DEBUG_FORCE_TIMEOUT = 1
DEBUG_TIME_KERNELS = 2
TIMER_SPLAT_FWD, TIMER_SPLAT_BWD, TIMER_FFT, TIMER_ENCODE, TIMER_TOTAL = 0, 1, 2, 3, 4
MAX_LAMBDA, MAX_SCENES = 16, 128

STATUS = {0: "GWS_OK", 1: "GWS_ERR_INVALID_ARG", 2: "GWS_ERR_WORKSPACE", 3: "GWS_ERR_CUDA",
          4: "GWS_ERR_NONFINITE", 5: "GWS_ERR_TIMEOUT", 6: "GWS_ERR_UNSUPPORTED", 7: "GWS_ERR_BOUNDS"}


class GwsError(RuntimeError):
    def __init__(self, code: int, where: str):
        super().__init__(f"{where}: {STATUS.get(code, code)}")
        self.code = code


class _Gaussians(C.Structure):
    _fields_ = [("mean", C.c_void_p), ("quat", C.c_void_p), ("scale", C.c_void_p), ("opacity", C.c_void_p),
                ("amp", C.c_void_p)]


class _Slm(C.Structure):
    _fields_ = [("H", C.c_int), ("W", C.c_int), ("pitch_x", C.c_double), ("pitch_y", C.c_double),
                ("n_lambda", C.c_int), ("wavelengths", C.POINTER(C.c_double))]


class _Opts(C.Structure):
    _fields_ = [("blend", C.c_int), ("prec", C.c_int), ("domain", C.c_int), ("phase_match", C.c_int),
                ("trunc_eps", C.c_float), ("alpha_min", C.c_float), ("tile_cfg", C.c_int),
                ("debug_flags", C.c_uint32), ("timeout_cycles", C.c_uint64), ("stream", C.c_void_p),
                ("workspace", C.c_void_p), ("workspace_bytes", C.c_size_t), ("t_binarize", C.c_float),
                ("exact_batch", C.c_int), ("pc_l", C.c_int), ("pc_m", C.c_int), ("pc_seed", C.c_uint64),
                ("pc_frame", C.c_uint64), ("pc_frames", C.c_int)]


class _GaussiansOut(C.Structure):
    _fields_ = [("mean", C.c_void_p), ("quat", C.c_void_p), ("scale", C.c_void_p), ("opacity", C.c_void_p),
                ("amp", C.c_void_p)]


class _Triangles(C.Structure):
    _fields_ = [("vertices", C.c_void_p), ("opacity", C.c_void_p), ("amp", C.c_void_p)]


class _WorldGaussians(C.Structure):
    _fields_ = [("mean", C.c_void_p), ("quat", C.c_void_p), ("scale", C.c_void_p), ("sh_opacity", C.c_void_p),
                ("opacity", C.c_void_p), ("sh_degree", C.c_int), ("sh_stride", C.c_int)]


class _Camera(C.Structure):
    _fields_ = [("view", C.c_double * 12), ("fx", C.c_double), ("fy", C.c_double), ("cx", C.c_double),
                ("cy", C.c_double), ("projection", C.c_int), ("z_near", C.c_double)]


_libs = {}
_variant = ""  # "" = libgws.so; "check" = libgws_check.so (bounds-checking build, tests only)
_lib_lock = threading.Lock()

EXPORTS = ["gws_opts_default", "gws_status_string", "gws_version", "gws_workspace_size", "gws_prepare",
           "gws_forward", "gws_forward_batched", "gws_backward", "gws_encode", "gws_get_device_status",
           "gws_depth_order", "gws_transmittance", "gws_footprints", "gws_last_launch_count", "gws_autotune",
           "gws_kernel_time_ms", "gws_footprint_pairs", "gws_encode_noalloc", "gws_holographics",
           "gws_triangles_workspace_size", "gws_forward_triangles", "gws_tile_config", "gws_tile_config_ext",
           "gws_tune_get", "gws_tune_set"]


def lib_path(variant: str | None = None) -> str:
    return _build.VARIANTS[_variant if variant is None else variant][0]


def load(build_if_needed: bool = True):
    """Loads libgws.so (building it in-tree first if sources are newer); inside ``checking_build()``
    the bounds-checking variant libgws_check.so instead."""
    with _lib_lock:
        lib = _libs.get(_variant)
        if lib is not None:
            return lib
        path = lib_path()
        if build_if_needed and _build.stale(_variant):
            _build.build(variants=(_variant,))
        if not os.path.exists(path):
            raise RuntimeError(f"{os.path.basename(path)} is not built; run __graft_entry__.build()")
        lib = C.CDLL(path)
        for name in EXPORTS:
            getattr(lib, name)  # raises AttributeError if an export is missing
        lib.gws_status_string.restype = C.c_char_p
        lib.gws_version.restype = C.c_int
        lib.gws_last_launch_count.restype = C.c_int
        lib.gws_kernel_time_ms.restype = C.c_float
        lib.gws_tile_config.restype = C.c_int
        lib.gws_tile_config_ext.restype = C.c_int
        for name in EXPORTS:
            if name not in ("gws_status_string", "gws_version", "gws_last_launch_count", "gws_opts_default",
                            "gws_kernel_time_ms", "gws_tile_config", "gws_tile_config_ext"):
                getattr(lib, name).restype = C.c_int
        _libs[_variant] = lib
        return lib


@contextlib.contextmanager
def checking_build():
    """Routes every call of this module to libgws_check.so (built with GWS_CHECK_BOUNDS: index checks
    in the kernels, canary words after the workspace's sub-buffers; a violation reads back as
    GWS_ERR_BOUNDS from gws_get_device_status).  For tests; not thread-safe."""
    global _variant
    old = _variant
    _variant = "check"
    try:
        yield load()
    finally:
        _variant = old


def _check(code: int, where: str):
    if code != 0:
        raise GwsError(code, where)


@dataclass
class Slm:
    H: int
    W: int
    pitch_x: float
    pitch_y: float
    wavelengths: tuple

    @property
    def n_lambda(self):
        return len(self.wavelengths)

    @classmethod
    def of(cls, s) -> "Slm":
        return cls(int(s.H), int(s.W), float(s.pitch_x), float(s.pitch_y), tuple(float(w) for w in s.wavelengths))

    def _c(self):
        wl = (C.c_double * len(self.wavelengths))(*self.wavelengths)
        st = _Slm(self.H, self.W, self.pitch_x, self.pitch_y, len(self.wavelengths), wl)
        st._keep = wl
        return st


@dataclass
class Gaussians:
    """Device tensors of one scene (structure of arrays, layouts of include/gws.h)."""
    mean: torch.Tensor     # float64 [n,3]
    quat: torch.Tensor     # float32 [n,4]
    scale: torch.Tensor    # float32 [n,2]
    opacity: torch.Tensor  # float32 [n]
    amp: torch.Tensor      # float32 [n,L]

    @property
    def n(self):
        return int(self.mean.shape[0])

    @classmethod
    def from_scene(cls, scene, device="cuda"):
        def t(a, dt):
            return torch.as_tensor(np.ascontiguousarray(a), dtype=dt, device=device)
        return cls(t(scene.mean, torch.float64), t(scene.quat, torch.float32), t(scene.scale, torch.float32),
                   t(scene.opacity, torch.float32), t(scene.amp, torch.float32))

    def check(self, n_lambda: int):
        n = self.n
        for name, t, dt, shape in (("mean", self.mean, torch.float64, (n, 3)), ("quat", self.quat, torch.float32, (n, 4)),
                                   ("scale", self.scale, torch.float32, (n, 2)),
                                   ("opacity", self.opacity, torch.float32, (n,)),
                                   ("amp", self.amp, torch.float32, (n, n_lambda))):
            if t.dtype != dt or tuple(t.shape) != shape or not t.is_contiguous() or not t.is_cuda:
                raise ValueError(f"{name}: expected contiguous CUDA {dt} {shape}, got {t.dtype} {tuple(t.shape)}")

    def _c(self):
        return _Gaussians(self.mean.data_ptr(), self.quat.data_ptr(), self.scale.data_ptr(),
                          self.opacity.data_ptr(), self.amp.data_ptr())


class _Workspace:
    """Grow-only per-device workspace (caller-owned scratch of the C ABI)."""

    def __init__(self):
        self.buf = {}

    def get(self, nbytes: int, device) -> torch.Tensor:
        dev = torch.device(device)
        key = dev.index if dev.index is not None else torch.cuda.current_device()
        b = self.buf.get(key)
        if b is None or b.numel() < nbytes:
            b = torch.empty(max(nbytes, 256), dtype=torch.uint8, device=dev)
            self.buf[key] = b
        return b


_WS = _Workspace()


def make_opts(blend=BLEND_OIT, prec=PREC_MIXED, domain=DOMAIN_FIELD, phase_match=False, trunc_eps=1e-5,
              alpha_min=1.0 / 255.0, tile_cfg=0, debug_flags=0, timeout_cycles=2_000_000_000, stream=None,
              t_binarize=0.0, exact_batch=0, pc_l=0, pc_m=0, pc_seed=0, pc_frame=0, pc_frames=0):
    lib = load()
    o = _Opts()
    lib.gws_opts_default(C.byref(o))
    o.blend, o.prec, o.domain, o.phase_match = int(blend), int(prec), int(domain), int(bool(phase_match))
    o.trunc_eps, o.alpha_min, o.tile_cfg = float(trunc_eps), float(alpha_min), int(tile_cfg)
    o.debug_flags, o.timeout_cycles = int(debug_flags), int(timeout_cycles)
    o.t_binarize, o.exact_batch = float(t_binarize), int(exact_batch)
    o.pc_l, o.pc_m, o.pc_seed, o.pc_frame = int(pc_l), int(pc_m), int(pc_seed), int(pc_frame)
    o.pc_frames = int(pc_frames)
    if stream is None:
        stream = torch.cuda.current_stream()
    o.stream = C.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))
    return o


def workspace_size(ns, slm: Slm, opts) -> int:
    lib = load()
    arr = (C.c_int64 * len(ns))(*ns)
    out = C.c_size_t(0)
    _check(lib.gws_workspace_size(arr, len(ns), C.byref(slm._c()), C.byref(opts), C.byref(out)), "gws_workspace_size")
    return int(out.value)


def _attach_ws(opts, ns, slm, device, workspace=None):
    nbytes = workspace_size(ns, slm, opts)
    ws = workspace if workspace is not None else _WS.get(nbytes, device)
    if ws.numel() < nbytes:
        raise GwsError(2, "workspace too small")
    opts.workspace = C.c_void_p(ws.data_ptr())
    opts.workspace_bytes = ws.numel()
    return ws


def prepare(slm: Slm, n_scenes=1, **kw):
    lib = load()
    opts = make_opts(**kw)
    _check(lib.gws_prepare(C.byref(slm._c()), C.byref(opts), int(n_scenes)), "gws_prepare")


def forward(g: Gaussians, slm: Slm, out: torch.Tensor | None = None, workspace=None, **kw) -> torch.Tensor:
    """u_SLM field (or spectrum with domain=DOMAIN_SPECTRUM), complex [L,H,W]; with
    blend=BLEND_PARTIAL_COHERENT and pc_frames=F > 1, the F frames' fields [F,L,H,W]."""
    lib = load()
    slm = Slm.of(slm)
    g.check(slm.n_lambda)
    opts = make_opts(**kw)
    dt = torch.complex128 if opts.prec == PREC_FP64 else torch.complex64
    frames = opts.pc_frames if opts.blend == BLEND_PARTIAL_COHERENT and opts.pc_frames > 1 else 0
    shape = ((frames,) if frames else ()) + (slm.n_lambda, slm.H, slm.W)
    if out is None:
        out = torch.empty(shape, dtype=dt, device=g.mean.device)
    elif out.numel() < math.prod(shape) or not out.is_contiguous():
        raise GwsError(1, f"out must be a contiguous tensor of at least {shape}")
    ws = _attach_ws(opts, [g.n], slm, g.mean.device, workspace)
    _check(lib.gws_forward(C.byref(g._c()), C.c_int64(g.n), C.byref(slm._c()), C.byref(opts),
                           C.c_void_p(out.data_ptr())), "gws_forward")
    out._gws_ws = ws  # keep the workspace alive while the stream uses it
    return out


def forward_batched(scenes, slm: Slm, outs=None, workspace=None, **kw):
    lib = load()
    slm = Slm.of(slm)
    for g in scenes:
        g.check(slm.n_lambda)
    opts = make_opts(**kw)
    dt = torch.complex128 if opts.prec == PREC_FP64 else torch.complex64
    dev = scenes[0].mean.device
    if outs is None:
        outs = [torch.empty((slm.n_lambda, slm.H, slm.W), dtype=dt, device=dev) for _ in scenes]
    ns = [g.n for g in scenes]
    ws = _attach_ws(opts, ns, slm, dev, workspace)
    arr = (_Gaussians * len(scenes))(*[g._c() for g in scenes])
    narr = (C.c_int64 * len(scenes))(*ns)
    parr = (C.c_void_p * len(scenes))(*[o.data_ptr() for o in outs])
    _check(lib.gws_forward_batched(arr, narr, len(scenes), C.byref(slm._c()), C.byref(opts), parr),
           "gws_forward_batched")
    return outs


def backward(g: Gaussians, slm: Slm, grad_field: torch.Tensor, workspace=None, **kw):
    """dL/d(mean, quat, scale, opacity, amp) given dL/d(field) (PyTorch complex convention)."""
    lib = load()
    slm = Slm.of(slm)
    g.check(slm.n_lambda)
    opts = make_opts(**kw)
    grad_field = grad_field.contiguous()
    out = {"mean": torch.empty_like(g.mean), "quat": torch.empty_like(g.quat), "scale": torch.empty_like(g.scale),
           "opacity": torch.empty_like(g.opacity), "amp": torch.empty_like(g.amp)}
    gg = _Gaussians(out["mean"].data_ptr(), out["quat"].data_ptr(), out["scale"].data_ptr(),
                    out["opacity"].data_ptr(), out["amp"].data_ptr())
    ws = _attach_ws(opts, [g.n], slm, g.mean.device, workspace)
    _check(lib.gws_backward(C.byref(g._c()), C.c_int64(g.n), C.byref(slm._c()), C.byref(opts),
                            C.c_void_p(grad_field.data_ptr()), C.byref(gg)), "gws_backward")
    out["_ws"] = ws
    return out


def encode(field: torch.Tensor, slm: Slm, amp_scale: float = 0.0, out=None, workspace=None, **kw) -> torch.Tensor:
    lib = load()
    slm = Slm.of(slm)
    kw.setdefault("prec", PREC_FP64 if field.dtype == torch.complex128 else PREC_MIXED)
    opts = make_opts(**kw)
    field = field.contiguous()
    if out is None:
        out = torch.empty((slm.n_lambda, slm.H, slm.W), dtype=torch.float32, device=field.device)
    ws = workspace if workspace is not None else _WS.get(4096, field.device)
    opts.workspace = C.c_void_p(ws.data_ptr())
    opts.workspace_bytes = ws.numel()
    _check(lib.gws_encode(C.c_void_p(field.data_ptr()), C.byref(slm._c()), C.byref(opts),
                          C.c_void_p(out.data_ptr()), C.c_float(amp_scale)), "gws_encode")
    return out


def encode_noalloc(field: torch.Tensor, slm: Slm, amp_scale: float = 0.0, out=None, **kw) -> torch.Tensor:
    """gws_encode_noalloc: the same encoding without a caller workspace (fixed in-library scratch)."""
    lib = load()
    slm = Slm.of(slm)
    kw.setdefault("prec", PREC_FP64 if field.dtype == torch.complex128 else PREC_MIXED)
    opts = make_opts(**kw)
    field = field.contiguous()
    if out is None:
        out = torch.empty((slm.n_lambda, slm.H, slm.W), dtype=torch.float32, device=field.device)
    _check(lib.gws_encode_noalloc(C.c_void_p(field.data_ptr()), C.byref(slm._c()), C.byref(opts),
                                  C.c_void_p(out.data_ptr()), C.c_float(amp_scale)), "gws_encode_noalloc")
    return out


def device_status(ns, slm: Slm, workspace=None, **kw) -> int:
    """Reads and clears the device status word of the shared workspace."""
    lib = load()
    slm = Slm.of(slm)
    opts = make_opts(**kw)
    dev = torch.device("cuda", torch.cuda.current_device())
    _attach_ws(opts, ns, slm, dev, workspace)
    return int(lib.gws_get_device_status(C.byref(opts)))


def depth_order(g: Gaussians, workspace=None, **kw) -> torch.Tensor:
    lib = load()
    opts = make_opts(**kw)
    out = torch.empty(g.n, dtype=torch.int32, device=g.mean.device)
    _attach_ws(opts, [g.n], Slm(1, 1, 1e-6, 1e-6, (5e-7,)), g.mean.device, workspace)
    _check(lib.gws_depth_order(C.byref(g._c()), C.c_int64(g.n), C.byref(opts), C.c_void_p(out.data_ptr())),
           "gws_depth_order")
    return out


def transmittance(g: Gaussians, workspace=None, **kw) -> torch.Tensor:
    lib = load()
    opts = make_opts(**kw)
    out = torch.empty(g.n, dtype=torch.float64, device=g.mean.device)
    _attach_ws(opts, [g.n], Slm(1, 1, 1e-6, 1e-6, (5e-7,)), g.mean.device, workspace)
    _check(lib.gws_transmittance(C.byref(g._c()), C.c_int64(g.n), C.byref(opts), C.c_void_p(out.data_ptr())),
           "gws_transmittance")
    return out


def footprints(g: Gaussians, slm: Slm, l: int = 0, workspace=None, **kw) -> torch.Tensor:
    lib = load()
    slm = Slm.of(slm)
    opts = make_opts(**kw)
    out = torch.empty((g.n, 3), dtype=torch.float32, device=g.mean.device)
    _attach_ws(opts, [g.n], slm, g.mean.device, workspace)
    _check(lib.gws_footprints(C.byref(g._c()), C.c_int64(g.n), C.byref(slm._c()), C.byref(opts), int(l),
                              C.c_void_p(out.data_ptr())), "gws_footprints")
    return out


def kernel_time_ms(which: int) -> float:
    """CUDA-event time of a timer of the last call made with debug_flags=DEBUG_TIME_KERNELS."""
    return float(load().gws_kernel_time_ms(int(which)))


def footprint_pairs(g: Gaussians, slm: Slm, workspace=None, **kw) -> int:
    """Algorithmic (Gaussian, wavelength, frequency) pairs inside the truncated footprints."""
    lib = load()
    slm = Slm.of(slm)
    opts = make_opts(**kw)
    _attach_ws(opts, [g.n], slm, g.mean.device, workspace)
    out = C.c_ulonglong(0)
    _check(lib.gws_footprint_pairs(C.byref(g._c()), C.c_int64(g.n), C.byref(slm._c()), C.byref(opts), C.byref(out)),
           "gws_footprint_pairs")
    return int(out.value)


def tune_cache_key(device_name: str, slm: Slm) -> str:
    """Key of a grid class in an autotuner cache file: the device, the library's configuration
    count (a build with another search space tunes again) and H x W x n_lambda."""
    slm = Slm.of(slm)
    n = int(load().gws_tile_config(0, None))
    return f"{device_name}|{n} configs|{slm.H}x{slm.W}x{slm.n_lambda}"


def _read_cache(path: str) -> dict:
    try:
        with open(path) as f:
            d = json.load(f)
        return d if isinstance(d, dict) else {}
    except (OSError, ValueError):
        return {}


def tuned(slm: Slm) -> int:
    """The configuration the library's autotuner table holds for this grid class (0: none)."""
    lib = load()
    c = C.c_int(0)
    _check(lib.gws_tune_get(C.byref(Slm.of(slm)._c()), C.byref(c)), "gws_tune_get")
    return int(c.value)


def load_tuned(cache: str, device_name: str, slm: Slm) -> int:
    """Restores a choice recorded in the JSON file ``cache`` for this device and grid class into
    the library's table (gws_tune_set) and returns it; 0 if the file has none (or an id the
    library does not have)."""
    lib = load()
    slm = Slm.of(slm)
    c = _read_cache(cache).get(tune_cache_key(device_name, slm))
    if not isinstance(c, int) or not 1 <= c <= int(lib.gws_tile_config(0, None)):
        return 0
    _check(lib.gws_tune_set(C.byref(slm._c()), C.c_int(c)), "gws_tune_set")
    return c


def store_tuned(cache: str, device_name: str, slm: Slm, cfg: int) -> None:
    """Adds (or replaces) this device's and grid class's choice in the JSON file ``cache``
    (written to a temporary file beside it, then renamed over it, so a reader never sees half a
    file; of two processes storing at once, the later one's file wins)."""
    d = _read_cache(cache)
    d[tune_cache_key(device_name, slm)] = int(cfg)
    folder = os.path.dirname(os.path.abspath(cache))
    os.makedirs(folder, exist_ok=True)
    fd, tmp = tempfile.mkstemp(prefix=".gws_tune_", dir=folder)
    with os.fdopen(fd, "w") as f:
        json.dump(d, f, indent=1, sort_keys=True)
    os.replace(tmp, cache)


def autotune(g: Gaussians, slm: Slm, workspace=None, cache: str | None = None, **kw) -> int:
    """Times every splat tile configuration on this scene; the fastest becomes the default
    for this (H, W, n_lambda).  Returns its id.  With ``cache`` (a JSON file), a choice recorded
    there for this device and grid class is taken without timing, and a new one is recorded."""
    lib = load()
    slm = Slm.of(slm)
    g.check(slm.n_lambda)
    dev_name = torch.cuda.get_device_name(g.mean.device) if cache is not None else None
    if cache is not None:
        c = load_tuned(cache, dev_name, slm)
        if c:
            return c
    opts = make_opts(**kw)
    scratch = torch.empty((slm.n_lambda, slm.H, slm.W), dtype=torch.complex64, device=g.mean.device)
    _attach_ws(opts, [g.n], slm, g.mean.device, workspace)
    best = C.c_int(0)
    _check(lib.gws_autotune(C.byref(g._c()), C.c_int64(g.n), C.byref(slm._c()), C.byref(opts),
                            C.c_void_p(scratch.data_ptr()), C.byref(best)), "gws_autotune")
    if cache is not None:
        store_tuned(cache, dev_name, slm, int(best.value))
    return int(best.value)


def tile_configs() -> dict:
    """The splat configurations the autotuner searches: id -> description."""
    lib = load()
    n = int(lib.gws_tile_config(0, None))
    out = {}
    for i in range(1, n + 1):
        d = (C.c_int * 9)()
        lib.gws_tile_config_ext(i, d, 9)
        out[i] = dict(zip(("tile_w", "tile_h", "px_per_thread", "records_per_iteration", "records_per_chunk",
                           "ring_stages", "ctas_per_sm", "cos_pairs_on_fp32", "column_step"), list(d)))
    return out


def forward_triangles(vertices: torch.Tensor, opacity: torch.Tensor, amp: torch.Tensor, slm: Slm,
                      out: torch.Tensor | None = None, workspace=None, **kw) -> torch.Tensor:
    """Field (or spectrum) of triangles (gws_forward_triangles): vertices float64 [n,3,3] (rows
    v1, v2, v3), opacity float32 [n], amp float32 [n,L], all contiguous CUDA tensors."""
    lib = load()
    n = int(vertices.shape[0])
    for name, t, dt, shape in (("vertices", vertices, torch.float64, (n, 3, 3)), ("opacity", opacity, torch.float32, (n,)),
                               ("amp", amp, torch.float32, (n, slm.n_lambda))):
        if t.dtype != dt or tuple(t.shape) != shape or not t.is_contiguous() or not t.is_cuda:
            raise ValueError(f"{name}: expected contiguous CUDA {dt} {shape}, got {t.dtype} {tuple(t.shape)}")
    dev = vertices.device
    if out is None:
        out = torch.empty((slm.n_lambda, slm.H, slm.W), dtype=torch.complex64, device=dev)
    opts = make_opts(**kw)
    nbytes = C.c_size_t(0)
    sc = slm._c()
    _check(lib.gws_triangles_workspace_size(C.c_int64(n), C.byref(sc), C.byref(opts), C.byref(nbytes)),
           "gws_triangles_workspace_size")
    ws = workspace if workspace is not None else _WS.get(int(nbytes.value), dev)
    if ws.numel() < nbytes.value:
        raise GwsError(2, "workspace too small")
    opts.workspace, opts.workspace_bytes = C.c_void_p(ws.data_ptr()), ws.numel()
    tri = _Triangles(vertices.data_ptr(), opacity.data_ptr(), amp.data_ptr())
    _check(lib.gws_forward_triangles(C.byref(tri), C.c_int64(n), C.byref(sc), C.byref(opts),
                                     C.c_void_p(out.data_ptr())), "gws_forward_triangles")
    return out


@dataclass
class WorldGaussians:
    """World-space Gaussians of a 2DGS / 2DGS-OIT style model (device tensors)."""
    mean: torch.Tensor                      # float64 [n,3]
    quat: torch.Tensor                      # float32 [n,4] (w, x, y, z)
    scale: torch.Tensor                     # float32 [n,3] (surfels: scale[:, 2] = 0)
    amp: torch.Tensor                       # float32 [n,L], passed through to the hologram-space set
    sh_opacity: torch.Tensor | None = None  # float32 [n,K], K >= (sh_degree + 1)^2
    opacity: torch.Tensor | None = None     # float32 [n], used when sh_opacity is None
    sh_degree: int = 3

    @property
    def n(self):
        return int(self.mean.shape[0])

    def check(self):
        n = self.n
        need = [("mean", self.mean, torch.float64, (n, 3)), ("quat", self.quat, torch.float32, (n, 4)),
                ("scale", self.scale, torch.float32, (n, 3))]
        if self.sh_opacity is not None:
            if self.sh_opacity.dim() != 2 or self.sh_opacity.shape[0] != n:
                raise ValueError("sh_opacity: expected [n, K]")
            need.append(("sh_opacity", self.sh_opacity, torch.float32, tuple(self.sh_opacity.shape)))
        elif self.opacity is not None:
            need.append(("opacity", self.opacity, torch.float32, (n,)))
        else:
            raise ValueError("either sh_opacity or opacity is required")
        for name, t, dt, shape in need:
            if t.dtype != dt or tuple(t.shape) != shape or not t.is_contiguous() or not t.is_cuda:
                raise ValueError(f"{name}: expected contiguous CUDA {dt} {shape}, got {t.dtype} {tuple(t.shape)}")


@dataclass
class Camera:
    """View [W | t] (3x4, x_view = W x_world + t, looking down -z) and projective mapping."""
    view: np.ndarray
    fx: float
    fy: float
    cx: float
    cy: float
    projection: int = PROJ_PERSPECTIVE
    z_near: float = 0.0

    def _c(self):
        v = np.ascontiguousarray(np.asarray(self.view, dtype=np.float64).reshape(12))
        return _Camera((C.c_double * 12)(*v.tolist()), float(self.fx), float(self.fy), float(self.cx), float(self.cy),
                       int(self.projection), float(self.z_near))


def holographics(world: WorldGaussians, camera: Camera, holo, compact: bool = True, stream=None):
    """Holographics front end (gws_holographics): world-space Gaussians -> the splat's
    hologram-space Gaussians for one view.  holo: 3x4 [A | b] (ray space -> hologram space).
    Returns (Gaussians, valid): with compact=True the culled Gaussians are dropped (valid then
    says which inputs were kept); otherwise every input keeps its slot."""
    world.check()
    lib = load()
    n, dev = world.n, world.mean.device
    mean = torch.empty((n, 3), dtype=torch.float64, device=dev)
    quat = torch.empty((n, 4), dtype=torch.float32, device=dev)
    scale = torch.empty((n, 2), dtype=torch.float32, device=dev)
    opacity = torch.empty((n,), dtype=torch.float32, device=dev)
    valid = torch.empty((n,), dtype=torch.uint8, device=dev)
    sh = world.sh_opacity
    win = _WorldGaussians(world.mean.data_ptr(), world.quat.data_ptr(), world.scale.data_ptr(),
                          sh.data_ptr() if sh is not None else None,
                          world.opacity.data_ptr() if (sh is None and world.opacity is not None) else None,
                          int(world.sh_degree), int(sh.shape[1]) if sh is not None else 0)
    out = _GaussiansOut(mean.data_ptr(), quat.data_ptr(), scale.data_ptr(), opacity.data_ptr(), None)
    h = np.ascontiguousarray(np.asarray(holo, dtype=np.float64).reshape(12))
    hc = (C.c_double * 12)(*h.tolist())
    opts = make_opts(stream=stream)
    _check(lib.gws_holographics(C.byref(win), C.c_int64(n), C.byref(camera._c()), hc, C.byref(opts), C.byref(out),
                                C.c_void_p(valid.data_ptr())), "gws_holographics")
    g = Gaussians(mean, quat, scale, opacity, world.amp)
    if compact:
        keep = valid.bool()
        g = Gaussians(mean[keep].contiguous(), quat[keep].contiguous(), scale[keep].contiguous(),
                      opacity[keep].contiguous(), world.amp[keep].contiguous())
    return g, valid


def last_launch_count() -> int:
    return int(load().gws_last_launch_count())


def status_string(code: int) -> str:
    return load().gws_status_string(int(code)).decode()


class GWSFunction(torch.autograd.Function):
    """field = GWS(mean, quat, scale, opacity, amp); backward through gws_backward."""

    @staticmethod
    def forward(ctx, mean, quat, scale, opacity, amp, slm, kw):
        g = Gaussians(mean.detach().contiguous(), quat.detach().contiguous(), scale.detach().contiguous(),
                      opacity.detach().contiguous(), amp.detach().contiguous())
        ctx.g, ctx.slm, ctx.kw = g, slm, dict(kw)
        return forward(g, slm, **kw)

    @staticmethod
    def backward(ctx, grad_field):
        gr = backward(ctx.g, ctx.slm, grad_field.contiguous(), **ctx.kw)
        return gr["mean"], gr["quat"], gr["scale"], gr["opacity"], gr["amp"], None, None


def gws_field(mean, quat, scale, opacity, amp, slm, **kw):
    return GWSFunction.apply(mean, quat, scale, opacity, amp, slm, kw)
