"""The bounds-checking build (libgws_check.so, GWS_CHECK_BOUNDS) on small cases of every entry point.

It stands in for a memory checker: its kernels check their tile, list and record indices (an
index out of range is recorded in the device status word and its access skipped) and its
workspace carries canary words after every sub-buffer, verified at the end of each call.  Each
case below (N <= 64 Gaussians, grids up to 64 x 80, ragged tiles) must leave the status word
clean (GWS_OK, not GWS_ERR_BOUNDS) and give the product build's results (or the oracle's)."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2505_06582_gb300 import gws
from paper_2505_06582_gb300.scenes import SLM, cotangent, random_field, surface_scene, triangle_scene, uniform_scene, \
    world_scene
from tests.helpers import rel_l2

pytestmark = pytest.mark.gpu

RGB = (638e-9, 520e-9, 450e-9)
SLM_A = SLM(32, 32, 8e-6, 8e-6, (520e-9,))
SLM_B = SLM(45, 70, 8e-6, 6e-6, RGB)  # ragged against every tile shape


def dev(sc):
    return gws.Gaussians.from_scene(sc, "cuda")


def _ws():
    return torch.empty(64 << 20, dtype=torch.uint8, device="cuda")


def _clean(ws, ns, slm, **kw):
    torch.cuda.synchronize()
    st = gws.device_status(ns, slm, workspace=ws, **kw)
    assert st == 0, gws.STATUS.get(st, st)


@pytest.fixture
def check():
    with gws.checking_build() as lib:
        yield lib


@pytest.mark.parametrize("slm,kind,n", [(SLM_A, "uniform", 64), (SLM_B, "surface", 50)])
@pytest.mark.parametrize("blend", [gws.BLEND_OIT, gws.BLEND_SORTED_T])
def test_forward_backward_clean_under_checks(check, slm, kind, n, blend):
    sc = (uniform_scene if kind == "uniform" else surface_scene)(5, n, slm)
    S = gws.Slm.of(slm)
    ws = _ws()
    ref = O.field(sc, slm, blend=blend)
    for prec, tol in ((gws.PREC_MIXED, 2e-4), (gws.PREC_FP64, 1e-6)):
        u = gws.forward(dev(sc), S, workspace=ws, prec=prec, blend=blend).cpu().numpy()
        _clean(ws, [n], S, prec=prec, blend=blend)
        assert rel_l2(u, ref) < tol
    G = cotangent(3, slm)
    gr = gws.backward(dev(sc), S, torch.as_tensor(G, device="cuda"), workspace=ws, blend=blend)
    _clean(ws, [n], S, blend=blend)
    gref = O.backward_field(sc, slm, G.astype(np.complex128), blend=blend)
    for k in ("mean", "quat", "scale", "opacity", "amp"):
        assert rel_l2(gr[k].cpu().numpy().astype(np.float64), gref[k]) < 2e-4, k


def test_every_tile_configuration_and_phase_match_clean(check):
    sc = surface_scene(6, 40, SLM_B)
    S = gws.Slm.of(SLM_B)
    ws = _ws()
    ref = O.field(sc, SLM_B, phase_match=True)
    for cfg in range(1, len(gws.tile_configs()) + 1):
        u = gws.forward(dev(sc), S, workspace=ws, tile_cfg=cfg, phase_match=True).cpu().numpy()
        _clean(ws, [sc.n], S)
        assert rel_l2(u, ref) < 2e-4, cfg


def test_batched_exact_partial_and_empty_clean(check):
    S = gws.Slm.of(SLM_B)
    ws = _ws()
    scenes = [surface_scene(10 + k, n, SLM_B) for k, n in enumerate((7, 0, 33, 12))]
    outs = gws.forward_batched([dev(s) for s in scenes], S, workspace=ws)
    _clean(ws, [s.n for s in scenes], S)
    for s, u in zip(scenes, outs):
        ref = O.field(s, SLM_B)
        if s.n == 0:
            assert np.all(u.cpu().numpy() == 0)
        else:
            assert rel_l2(u.cpu().numpy(), ref) < 2e-4
    sc = surface_scene(14, 20, SLM_B)
    for blend, kw in ((gws.BLEND_EXACT, dict(exact_batch=7)),
                      (gws.BLEND_PARTIAL_COHERENT, dict(pc_l=1, pc_m=-1, pc_seed=3, pc_frames=2, exact_batch=6))):
        gws.forward(dev(sc), S, workspace=ws, blend=blend, **kw)
        _clean(ws, [sc.n], S, blend=blend, **kw)
    assert rel_l2(gws.forward(dev(sc), S, workspace=ws, blend=gws.BLEND_EXACT, domain=gws.DOMAIN_SPECTRUM).cpu().numpy(),
                  O.exact_awb(sc, SLM_B)) < 2e-4
    _clean(ws, [sc.n], S, blend=gws.BLEND_EXACT, domain=gws.DOMAIN_SPECTRUM)


def test_inspection_encode_and_tuning_clean(check):
    sc = surface_scene(20, 48, SLM_B)
    S = gws.Slm.of(SLM_B)
    ws = _ws()
    g = dev(sc)
    assert np.array_equal(gws.depth_order(g, workspace=ws).cpu().numpy(), O.depth_order(sc.mean))
    _clean(ws, [sc.n], S)
    assert np.abs(gws.transmittance(g, workspace=ws).cpu().numpy() - O.transmittance(sc)).max() < 1e-12
    _clean(ws, [sc.n], S)
    gws.footprints(g, S, l=2, workspace=ws)
    _clean(ws, [sc.n], S)
    assert gws.footprint_pairs(g, S, workspace=ws) > 0
    _clean(ws, [sc.n], S)
    assert 1 <= gws.autotune(g, S, workspace=ws) <= len(gws.tile_configs())
    _clean(ws, [sc.n], S)
    f = torch.as_tensor(random_field(21, (3, SLM_B.H, SLM_B.W)).astype(np.complex64), device="cuda")
    p = gws.encode(f, S, workspace=ws).cpu().numpy()
    _clean(ws, [0], S)
    assert np.array_equal(gws.encode_noalloc(f, S).cpu().numpy(), p)


def test_triangles_and_front_end_match_the_product_build(check):
    verts, opa, amp = triangle_scene(30, 25, SLM_B, size_px=4.0)
    t = lambda a, dt: torch.as_tensor(np.ascontiguousarray(a), dtype=dt, device="cuda")
    S = gws.Slm.of(SLM_B)
    got = gws.forward_triangles(t(verts, torch.float64), t(opa, torch.float32), t(amp, torch.float32), S).cpu().numpy()
    w = world_scene(31, 64, SLM_B)
    wd = gws.WorldGaussians(t(w.mean, torch.float64), t(w.quat, torch.float32), t(w.scale, torch.float32),
                            t(w.amp, torch.float32), sh_opacity=t(w.sh, torch.float32), sh_degree=3)
    cam = gws.Camera(w.view, w.fx, w.fy, w.cx, w.cy, gws.PROJ_PERSPECTIVE, 0.1)
    gh, valid = gws.holographics(wd, cam, w.holo, compact=False)
    gh = {k: getattr(gh, k).cpu().numpy() for k in ("mean", "quat", "scale", "opacity")}
    valid = valid.cpu().numpy()
    torch.cuda.synchronize()
    gws._variant = ""  # the product build, same inputs
    try:
        ref = gws.forward_triangles(t(verts, torch.float64), t(opa, torch.float32), t(amp, torch.float32),
                                    S).cpu().numpy()
        gp, vp = gws.holographics(wd, cam, w.holo, compact=False)
    finally:
        gws._variant = "check"
    assert rel_l2(got, ref) < 1e-6
    assert np.array_equal(valid, vp.cpu().numpy())
    for k in gh:
        assert np.allclose(gh[k], getattr(gp, k).cpu().numpy(), rtol=1e-6, atol=1e-12), k
