"""CPU checks of the C ABI: the library builds for sm_103a, loads, exports every symbol
include/gws.h declares, and rejects bad arguments on the host (no GPU calls)."""
import ctypes as C
import os
import re

import pytest

from paper_2505_06582_gb300 import _build, gws

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "gws.h")).read()
    return sorted(set(re.findall(r"^GWS_API [^(]*?\b(gws_\w+)\(", src, flags=re.M)))


def test_library_exports_every_declared_symbol():
    lib = gws.load()
    names = declared_functions()
    assert len(names) >= 15
    for n in names:
        assert hasattr(lib, n), n
    assert set(names) == set(gws.EXPORTS)


def test_library_is_built_for_sm_103a_only():
    out = os.popen(f"{_build.NVCC} --version").read()
    assert "release" in out
    assert _build.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]
    assert os.path.exists(_build.LIB)


def test_checking_build_exports_the_same_symbols_and_reserves_canaries():
    """libgws_check.so (GWS_CHECK_BOUNDS) is the same ABI; its workspace has canary words after every
    sub-buffer, so it asks for more bytes."""
    assert os.path.exists(_build.LIB_CHECK)
    chk = C.CDLL(_build.LIB_CHECK)
    for n in declared_functions():
        assert hasattr(chk, n), n
    wl = (C.c_double * 3)(6.38e-7, 5.2e-7, 4.5e-7)
    s = gws._Slm(45, 70, 8e-6, 6e-6, 3, wl)
    sizes = []
    for lib in (gws.load(), chk):
        o = gws._Opts()
        lib.gws_opts_default(C.byref(o))
        o.domain = 1  # spectrum: no FFT plan (no GPU call) in the size query
        arr = (C.c_int64 * 1)(64)
        out = C.c_size_t(0)
        assert lib.gws_workspace_size(arr, 1, C.byref(s), C.byref(o), C.byref(out)) == 0
        sizes.append(out.value)
    assert sizes[1] > sizes[0] + 40 * 64
    chk.gws_status_string.restype = C.c_char_p
    assert chk.gws_status_string(7).decode() == "GWS_ERR_BOUNDS"


def test_tile_configurations_are_described():
    """The autotuner's search space (tile shape, pixels per thread, records per iteration, records
    per chunk, ring depth, CTAs per SM): more than tile shapes alone, chunks within the CTA's threads."""
    cfgs = gws.tile_configs()
    assert len(cfgs) >= 8
    assert len({c["records_per_chunk"] for c in cfgs.values()}) >= 3
    assert len({c["ring_stages"] for c in cfgs.values()}) >= 3
    for c in cfgs.values():
        threads = c["tile_w"] // c["px_per_thread"] * c["tile_h"]
        assert 32 <= c["records_per_chunk"] <= min(threads, 256) and c["records_per_chunk"] % 32 == 0
    lib = gws.load()
    assert lib.gws_tile_config(0, None) == len(cfgs) and lib.gws_tile_config(99, None) == len(cfgs)
    # the extended description writes no more than it is given room for
    d = (C.c_int * 10)(*([-7] * 10))
    assert lib.gws_tile_config_ext(1, d, 3) == len(cfgs) and list(d)[3:] == [-7] * 7
    assert lib.gws_tile_config_ext(1, d, 10) == len(cfgs) and d[9] == -7 and d[8] in (0, 1)
    assert {c["column_step"] for c in cfgs.values()} == {0, 1}


def test_status_strings_and_version():
    lib = gws.load()
    assert lib.gws_version() == 1
    for code, name in gws.STATUS.items():
        assert lib.gws_status_string(code).decode() == name


def test_defaults():
    lib = gws.load()
    o = gws._Opts()
    lib.gws_opts_default(C.byref(o))
    assert (o.blend, o.prec, o.domain, o.phase_match) == (0, 1, 0, 0)
    assert abs(o.trunc_eps - 1e-5) < 1e-12 and abs(o.alpha_min - 1 / 255) < 1e-9
    assert o.timeout_cycles > 0 and not o.workspace


def _opts(**kw):
    lib = gws.load()
    o = gws._Opts()
    lib.gws_opts_default(C.byref(o))
    for k, v in kw.items():
        setattr(o, k, v)
    return o


@pytest.mark.parametrize("bad", [
    dict(H=0), dict(W=-1), dict(pitch_x=0.0), dict(pitch_y=float("nan")), dict(n_lambda=0), dict(n_lambda=17),
    dict(wl=-5e-7), dict(wl=float("inf")),
])
def test_bad_slm_rejected_on_host(bad):
    lib = gws.load()
    wl = (C.c_double * 16)(*([bad.get("wl", 5e-7)] * 16))
    s = gws._Slm(bad.get("H", 8), bad.get("W", 8), bad.get("pitch_x", 8e-6), bad.get("pitch_y", 8e-6),
                 bad.get("n_lambda", 1), wl)
    n = (C.c_int64 * 1)(4)
    out = C.c_size_t(0)
    o = _opts(domain=1)
    assert lib.gws_workspace_size(n, 1, C.byref(s), C.byref(o), C.byref(out)) == 1


@pytest.mark.parametrize("bad", [dict(blend=5), dict(prec=2), dict(domain=9), dict(trunc_eps=0.0),
                                 dict(trunc_eps=1.5), dict(alpha_min=-0.1), dict(timeout_cycles=0),
                                 dict(tile_cfg=99), dict(pc_frames=-1), dict(pc_frames=65)])
def test_bad_options_rejected_on_host(bad):
    lib = gws.load()
    wl = (C.c_double * 1)(5e-7)
    s = gws._Slm(8, 8, 8e-6, 8e-6, 1, wl)
    n = (C.c_int64 * 1)(4)
    out = C.c_size_t(0)
    o = _opts(domain=1)
    for k, v in bad.items():
        setattr(o, k, v)
    assert lib.gws_workspace_size(n, 1, C.byref(s), C.byref(o), C.byref(out)) == 1


def test_workspace_size_grows_with_n_and_covers_layout():
    lib = gws.load()
    wl = (C.c_double * 3)(6.38e-7, 5.2e-7, 4.5e-7)
    s = gws._Slm(64, 96, 8e-6, 8e-6, 3, wl)
    sizes = []
    for n in (0, 10, 1000, 100000):
        arr = (C.c_int64 * 1)(n)
        out = C.c_size_t(0)
        assert lib.gws_workspace_size(arr, 1, C.byref(s), C.byref(_opts(domain=1)), C.byref(out)) == 0
        sizes.append(out.value)
    assert sizes == sorted(sizes) and sizes[-1] > 100000 * 3 * 96
    # too many scenes / negative sizes
    arr = (C.c_int64 * 2)(5, -1)
    out = C.c_size_t(0)
    assert lib.gws_workspace_size(arr, 2, C.byref(s), C.byref(_opts(domain=1)), C.byref(out)) == 1
    assert lib.gws_workspace_size(arr, 0, C.byref(s), C.byref(_opts(domain=1)), C.byref(out)) == 1


def test_null_arguments_rejected_before_any_launch():
    lib = gws.load()
    wl = (C.c_double * 1)(5e-7)
    s = gws._Slm(8, 8, 8e-6, 8e-6, 1, wl)
    o = _opts(domain=1)
    g = gws._Gaussians(0, 0, 0, 0, 0)
    # null Gaussian arrays with n > 0
    assert lib.gws_forward(C.byref(g), C.c_int64(3), C.byref(s), C.byref(o), C.c_void_p(16)) == 1
    # null output
    assert lib.gws_forward(C.byref(g), C.c_int64(0), C.byref(s), C.byref(o), None) == 1
    # missing workspace
    ok = gws._Gaussians(256, 256, 256, 256, 256)
    assert lib.gws_forward(C.byref(ok), C.c_int64(3), C.byref(s), C.byref(o), C.c_void_p(256)) == 2
    # misaligned workspace
    o.workspace, o.workspace_bytes = C.c_void_p(256 + 8), 1 << 30
    assert lib.gws_forward(C.byref(ok), C.c_int64(3), C.byref(s), C.byref(o), C.c_void_p(256)) == 2
    # encode: null field
    assert lib.gws_encode(None, C.byref(s), C.byref(o), C.c_void_p(256), C.c_float(0)) == 1


@pytest.mark.parametrize("bad", [dict(amp=float("-inf")), dict(amp=float("nan")), dict(amp=float("inf")),
                                 dict(pitch_x=0.0), dict(wl=-5e-7), dict(blend=7), dict(prec=3), dict(trunc_eps=0.0),
                                 dict(field=None), dict(phase=None), dict(n_lambda=0), dict(H=0)])
def test_encode_entry_points_return_the_same_status_for_bad_arguments(bad):
    """gws_encode and gws_encode_noalloc share their argument checks (no GPU call is reached)."""
    lib = gws.load()
    wl = (C.c_double * 2)(*([bad.get("wl", 5e-7)] * 2))
    s = gws._Slm(bad.get("H", 8), 8, bad.get("pitch_x", 8e-6), 8e-6, bad.get("n_lambda", 2), wl)
    o = _opts()
    for k in ("blend", "prec", "trunc_eps"):
        if k in bad:
            setattr(o, k, bad[k])
    field = bad.get("field", 256)
    phase = bad.get("phase", 256)
    args = (C.c_void_p(field) if field else None, C.byref(s), C.byref(o), C.c_void_p(phase) if phase else None,
            C.c_float(bad.get("amp", 1.0)))
    a = lib.gws_encode(*args)
    b = lib.gws_encode_noalloc(*args)
    assert a == b == 1


def test_triangle_entry_points_check_arguments_on_host():
    lib = gws.load()
    wl = (C.c_double * 2)(6.38e-7, 4.5e-7)
    s = gws._Slm(32, 48, 8e-6, 8e-6, 2, wl)
    out = C.c_size_t(0)
    assert lib.gws_triangles_workspace_size(C.c_int64(10), C.byref(s), C.byref(_opts()), None) == 1
    assert lib.gws_triangles_workspace_size(C.c_int64(-1), C.byref(s), C.byref(_opts()), C.byref(out)) == 1
    assert lib.gws_triangles_workspace_size(C.c_int64(10), C.byref(s), C.byref(_opts(prec=0)), C.byref(out)) == 6
    sizes = []
    for n in (0, 100, 10000):  # spectrum domain: the size needs no cuFFT plan (no GPU here)
        assert lib.gws_triangles_workspace_size(C.c_int64(n), C.byref(s), C.byref(_opts(domain=1)),
                                                C.byref(out)) == 0
        sizes.append(out.value)
    assert sizes == sorted(sizes) and sizes[0] < sizes[-1]
    t = gws._Triangles(256, 256, 256)
    o = _opts(domain=1)
    assert lib.gws_forward_triangles(C.byref(t), C.c_int64(3), C.byref(s), C.byref(o), None) == 1
    null = gws._Triangles(0, 256, 256)
    assert lib.gws_forward_triangles(C.byref(null), C.c_int64(3), C.byref(s), C.byref(o), C.c_void_p(256)) == 1
    assert lib.gws_forward_triangles(C.byref(t), C.c_int64(3), C.byref(s), C.byref(o), C.c_void_p(256)) == 2
    o.workspace, o.workspace_bytes = C.c_void_p(256 + 16), 1 << 30
    assert lib.gws_forward_triangles(C.byref(t), C.c_int64(3), C.byref(s), C.byref(o), C.c_void_p(256)) == 2


def _camera(**kw):
    cam = gws._Camera()
    view = kw.get("view", [1, 0, 0, 0, 0, 1, 0, 0, 0, 0, 1, 0])
    for k in range(12):
        cam.view[k] = view[k]
    cam.fx, cam.fy, cam.cx, cam.cy = kw.get("fx", 500.0), 500.0, 320.0, 240.0
    cam.projection, cam.z_near = kw.get("projection", 0), 0.1
    return cam


@pytest.mark.parametrize("bad", [
    dict(sh_degree=4), dict(sh_degree=-1), dict(sh_degree=2, sh_stride=5), dict(projection=7),
    dict(view=[float("nan")] + [0.0] * 11), dict(fx=float("inf")),
    dict(holo=[0.0, 1, 0, 0, 0.0, 0, 1, 0, 0.0, 0, 0, 1]),       # A's first column zero
    dict(holo=[1.0, 2.0, 0, 0, 0.0, 0.0, 1, 0, 0.0, 0.0, 0, 1]),  # A's xy columns parallel
    dict(n=-1),
])
def test_holographics_checks_arguments_on_host(bad):
    lib = gws.load()
    w = gws._WorldGaussians(256, 256, 256, 256, 256, bad.get("sh_degree", 0), bad.get("sh_stride", 0))
    cam = _camera(**{k: v for k, v in bad.items() if k in ("view", "fx", "projection")})
    holo = (C.c_double * 12)(*bad.get("holo", [1e-5, 0, 0, 0, 0, 1e-5, 0, 0, 0, 0, 1e-3, 5e-3]))
    out = gws._GaussiansOut(256, 256, 256, 256, 256)
    st = lib.gws_holographics(C.byref(w), C.c_int64(bad.get("n", 4)), C.byref(cam), holo, C.byref(_opts()),
                              C.byref(out), C.c_void_p(256))
    assert st == 1


def test_holographics_rejects_null_pointers_on_host():
    lib = gws.load()
    w = gws._WorldGaussians(256, 256, 256, 256, 256, 0, 0)
    cam = _camera()
    holo = (C.c_double * 12)(1e-5, 0, 0, 0, 0, 1e-5, 0, 0, 0, 0, 1e-3, 5e-3)
    out = gws._GaussiansOut(256, 256, 256, 256, 256)
    args = [C.byref(w), C.c_int64(4), C.byref(cam), holo, C.byref(_opts()), C.byref(out), C.c_void_p(256)]
    for i in (0, 2, 3, 4, 5):
        a = list(args)
        a[i] = None
        assert lib.gws_holographics(*a) == 1, i


def test_struct_layouts_match_the_header(tmp_path):
    # every ctypes mirror in the binding has the C struct's field offsets and size (gcc on the header)
    pairs = [("gws_gaussians", gws._Gaussians), ("gws_slm", gws._Slm), ("gws_opts", gws._Opts),
             ("gws_gaussians_out", gws._GaussiansOut), ("gws_triangles", gws._Triangles),
             ("gws_world_gaussians", gws._WorldGaussians), ("gws_camera", gws._Camera)]
    lines = ["#include <stddef.h>", "#include <stdio.h>", '#include "gws.h"', "int main(void) {"]
    for cname, py in pairs:
        lines.append(f'    printf("{cname} size %zu\\n", sizeof({cname}));')
        for fname, _ in py._fields_:
            lines.append(f'    printf("{cname} {fname} %zu\\n", offsetof({cname}, {fname}));')
    lines += ["    return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    assert os.system(f"gcc -I{os.path.join(ROOT, 'include')} {src} -o {exe}") == 0
    got = {}
    for line in os.popen(str(exe)).read().splitlines():
        cname, field, value = line.split()
        got[(cname, field)] = int(value)
    for cname, py in pairs:
        assert got[(cname, "size")] == C.sizeof(py), cname
        for fname, _ in py._fields_:
            assert got[(cname, fname)] == getattr(py, fname).offset, (cname, fname)


def test_autotuner_table_and_its_cache_file(tmp_path):
    """gws_tune_set / gws_tune_get (host only) and the JSON cache that keeps choices between
    processes: a stored choice is restored into the library's table for the same device and
    grid class only; ids the library does not have, and unreadable files, restore nothing."""
    lib = gws.load()
    slm = gws.Slm(72, 88, 8e-6, 8e-6, (638e-9, 450e-9))
    other = gws.Slm(72, 88, 8e-6, 8e-6, (520e-9,))
    n = lib.gws_tile_config(0, None)
    assert gws.tuned(slm) == 0
    assert lib.gws_tune_set(C.byref(slm._c()), C.c_int(n + 1)) == 1
    assert lib.gws_tune_set(C.byref(slm._c()), C.c_int(-1)) == 1
    assert lib.gws_tune_get(C.byref(slm._c()), None) == 1
    assert lib.gws_tune_set(C.byref(slm._c()), C.c_int(n)) == 0 and gws.tuned(slm) == n
    assert gws.tuned(other) == 0
    assert lib.gws_tune_set(C.byref(slm._c()), C.c_int(0)) == 0 and gws.tuned(slm) == 0

    cache = str(tmp_path / "sub" / "tune.json")  # its folder is created on the first store
    assert gws.load_tuned(cache, "GPU A", slm) == 0  # no file yet
    gws.store_tuned(cache, "GPU A", slm, 2)
    gws.store_tuned(cache, "GPU A", other, 3)
    assert gws.load_tuned(cache, "GPU B", slm) == 0 and gws.tuned(slm) == 0  # another device
    assert gws.load_tuned(cache, "GPU A", slm) == 2 and gws.tuned(slm) == 2
    assert gws.load_tuned(cache, "GPU A", other) == 3 and gws.tuned(other) == 3
    with open(cache) as f:
        assert len(__import__("json").load(f)) == 2
    gws.store_tuned(cache, "GPU A", slm, n + 5)  # an id this build does not have
    assert gws.load_tuned(cache, "GPU A", slm) == 0
    with open(cache, "w") as f:
        f.write("{not json")
    assert gws.load_tuned(cache, "GPU A", slm) == 0
    for s in (slm, other):
        assert lib.gws_tune_set(C.byref(s._c()), C.c_int(0)) == 0
