"""GPU parity of the holographics front end and the SH view-dependent opacity (gws_holographics)
against the FP64 oracle (oracle/holographics.py).

Bars: the valid flags bit-exact (FP64 decisions on both sides; no input within 1e-9 of the
z_near boundary); the hologram-space mean (FP64 output) to 1e-12 of the scene extent; the
covariance Sigma = R diag(s_u^2, s_v^2, 0) R^T rebuilt from the float32 outputs to 2e-6 of its
largest entry; the scales to 1e-6 relative (float32 rounding); the opacity to 1e-6 (float32
output); the normal r3 parallel to the oracle's (the signs of r1, r2 are free).  Chain: the
splat of the front end's output against the oracle's spectrum of the oracle's front end.
"""
import numpy as np
import pytest
import torch

import oracle as O
from oracle import holographics as OH
from paper_2505_06582_gb300 import gws
from paper_2505_06582_gb300.scenes import SLM, Scene, world_scene
from tests.helpers import rel_l2

pytestmark = pytest.mark.gpu

RGB = (638e-9, 520e-9, 450e-9)


def world_dev(w, sh_degree=3, sh=None, opacity=None):
    t = lambda a, dt: torch.as_tensor(np.ascontiguousarray(a), dtype=dt, device="cuda")
    return gws.WorldGaussians(t(w.mean, torch.float64), t(w.quat, torch.float32), t(w.scale, torch.float32),
                              t(w.amp, torch.float32),
                              sh_opacity=None if opacity is not None else t(w.sh if sh is None else sh, torch.float32),
                              opacity=None if opacity is None else t(opacity, torch.float32), sh_degree=sh_degree)


def camera(w, proj=gws.PROJ_PERSPECTIVE, z_near=0.1):
    return gws.Camera(w.view, w.fx, w.fy, w.cx, w.cy, proj, z_near)


def oracle_front(w, proj=OH.PROJ_PERSPECTIVE, z_near=0.1, sh_degree=3, holo=None):
    out = OH.holographics(w.mean, w.quat.astype(np.float64), w.scale.astype(np.float64), w.view, w.fx, w.fy, w.cx,
                          w.cy, proj, z_near, w.holo if holo is None else holo)
    out["opacity"] = OH.view_opacity(w.sh.astype(np.float64), w.mean, w.view, sh_degree)
    return out


def sigma_of(quat, scale):
    R = OH.rotation(np.asarray(quat, dtype=np.float64))
    s = np.asarray(scale, dtype=np.float64)
    return np.einsum("nik,nk,njk->nij", R[:, :, :2], s ** 2, R[:, :, :2])


def compare(g, valid, ref, extent):
    v = valid.cpu().numpy().astype(bool)
    assert np.array_equal(v, ref["valid"] & (ref["scale"][:, 1] > 0))
    mean = g.mean.cpu().numpy()[v]
    assert np.abs(mean - ref["mean"][v]).max() <= 1e-12 * extent
    q, s = g.quat.cpu().numpy()[v], g.scale.cpu().numpy()[v]
    sig = sigma_of(q, s)
    ref_sig = ref["sigma"][v]
    big = np.abs(ref_sig).max(axis=(1, 2))
    assert np.all(np.abs(sig - ref_sig).max(axis=(1, 2)) <= 2e-6 * big)
    assert np.allclose(s, ref["scale"][v], rtol=1e-6, atol=0)
    assert np.all(s[:, 0] >= s[:, 1])
    assert np.allclose(np.linalg.norm(q, axis=1), 1.0, atol=1e-6) and np.all(q[:, 0] >= 0)
    n_gpu = OH.rotation(q.astype(np.float64))[:, :, 2]
    n_ref = OH.rotation(ref["quat"][v])[:, :, 2]
    assert np.all(np.abs(np.sum(n_gpu * n_ref, axis=1)) >= 1 - 1e-6)
    assert np.abs(g.opacity.cpu().numpy()[v] - ref["opacity"][v]).max() <= 1e-6


@pytest.mark.parametrize("seed,proj,volume_frac", [(0, gws.PROJ_PERSPECTIVE, 0.0), (1, gws.PROJ_PERSPECTIVE, 0.5),
                                                   (2, gws.PROJ_ORTHOGRAPHIC, 0.3)])
def test_front_parity(seed, proj, volume_frac):
    slm = SLM(1080, 1920, 8e-6, 8e-6, RGB)
    w = world_scene(seed, 5000, slm, volume_frac=volume_frac)
    if proj == gws.PROJ_ORTHOGRAPHIC:  # orthographic mapping with the same pixel scale at 2 m
        w.fx, w.fy = w.fx / 2.0, w.fy / 2.0
    g, valid = gws.holographics(world_dev(w), camera(w, proj), w.holo, compact=False)
    ref = oracle_front(w, proj)
    compare(g, valid, ref, extent=1e-2)


def test_front_general_hologram_transform_and_sh_stride():
    # a sheared, non-orthogonal A (the QR path) and SH rows wider than the degree needs
    rng = np.random.default_rng(7)
    slm = SLM(256, 256, 8e-6, 8e-6, (520e-9,))
    w = world_scene(3, 2000, slm, volume_frac=0.5)
    w.holo = w.holo.copy()
    w.holo[:, :3] = w.holo[:, :3] @ (np.eye(3) + 0.3 * rng.normal(size=(3, 3)))
    sh = np.concatenate([w.sh, rng.normal(size=(w.n, 5)).astype(np.float32)], axis=1)  # stride 21
    for deg in (0, 1, 2, 3):
        g, valid = gws.holographics(world_dev(w, deg, sh=sh), camera(w), w.holo, compact=False)
        ref = oracle_front(w, sh_degree=deg)
        compare(g, valid, ref, extent=1e-2)


def test_front_view_independent_opacity_passes_through():
    slm = SLM(128, 128, 8e-6, 8e-6, (520e-9,))
    w = world_scene(4, 500, slm)
    op = np.random.default_rng(1).uniform(0, 1, w.n).astype(np.float32)
    g, valid = gws.holographics(world_dev(w, opacity=op), camera(w), w.holo, compact=False)
    assert valid.bool().all()
    assert np.array_equal(g.opacity.cpu().numpy(), op)


def test_front_culling_and_degenerate_inputs():
    slm = SLM(128, 128, 8e-6, 8e-6, (520e-9,))
    w = world_scene(5, 64, slm)
    Rc, t = w.view[:, :3], w.view[:, 3]
    ctr = -Rc.T @ t
    fwd = -Rc[2]  # viewing direction in the world
    mean = w.mean.copy()
    quat = w.quat.copy()
    scale = w.scale.copy()
    mean[0] = ctr - 1.0 * fwd            # behind the camera
    mean[1] = ctr + 0.05 * fwd           # in front, but closer than z_near = 0.1
    mean[2] = ctr + 0.0 * fwd            # at the camera centre
    mean[3, 0] = np.nan                  # non-finite
    quat[4] = 0.0                        # zero-norm quaternion
    scale[5, 1] = -1e-3                  # negative scale
    # an edge-on surfel: its normal perpendicular to the viewing ray, so its projection is a line
    ray = (mean[6] - ctr) / np.linalg.norm(mean[6] - ctr)
    e1 = np.cross(ray, [0.0, 0.0, 1.0])
    e1 /= np.linalg.norm(e1)
    r1, r3 = ray, e1
    r2 = np.cross(r3, r1)
    from paper_2505_06582_gb300.scenes import _quat_from_frame
    quat[6] = _quat_from_frame(r1[None], r2[None], r3[None])[0]
    scale[6] = [2e-3, 1e-3, 0.0]  # the axis along the ray projects to a point: a line remains
    w2 = world_scene(5, 64, slm)
    w2.mean, w2.quat, w2.scale = mean, quat.astype(np.float32), scale
    g, valid = gws.holographics(world_dev(w2), camera(w2), w2.holo, compact=False)
    v = valid.cpu().numpy()
    assert v[:6].tolist() == [0, 0, 0, 0, 0, 0]
    assert v[7:].all()
    # the edge-on surfel keeps its slot with a vanishing width (weight ~ s_u s_v ~ 0), unless
    # the width rounds to zero in float32, when it is culled
    s6 = g.scale.cpu().numpy()[6]
    assert (v[6] == 1 and s6[1] <= 1e-6 * s6[0]) or (v[6] == 0 and s6[1] == 0)
    bad = ~v.astype(bool)
    assert np.all(g.scale.cpu().numpy()[bad] == 0) and np.all(g.opacity.cpu().numpy()[bad] == 0)
    assert np.all(g.mean.cpu().numpy()[bad] == 0)
    assert np.all(g.quat.cpu().numpy()[bad] == np.array([1, 0, 0, 0], np.float32))
    # compaction keeps exactly the valid ones, in order
    gc, _ = gws.holographics(world_dev(w2), camera(w2), w2.holo, compact=True)
    assert gc.n == int(v.sum())
    assert torch.equal(gc.mean, g.mean[valid.bool()])


def test_front_invalid_arguments():
    slm = SLM(64, 64, 8e-6, 8e-6, (520e-9,))
    w = world_scene(6, 16, slm)
    wd = world_dev(w)
    wd.sh_degree = 4
    with pytest.raises(gws.GwsError):
        gws.holographics(wd, camera(w), w.holo)
    wd = world_dev(w)
    flat = w.holo.copy()
    flat[:, 1] = 2.0 * flat[:, 0]  # A's xy columns parallel
    with pytest.raises(gws.GwsError):
        gws.holographics(wd, camera(w), flat)
    cam = camera(w)
    cam.projection = 7
    with pytest.raises(gws.GwsError):
        gws.holographics(wd, cam, w.holo)
    # empty input
    w0 = world_scene(6, 0, slm)
    g, valid = gws.holographics(world_dev(w0), camera(w0), w0.holo)
    assert g.n == 0 and valid.numel() == 0


def test_front_chain_into_the_splat():
    # world scene -> GPU front end -> GPU forward, against the oracle's front end -> oracle field
    slm = SLM(96, 128, 8e-6, 8e-6, (638e-9, 520e-9))
    w = world_scene(8, 120, slm, depth=(1.5, 3.0), scale_px=3.0)
    g, valid = gws.holographics(world_dev(w), camera(w), w.holo)
    assert valid.bool().all()
    field = gws.forward(g, gws.Slm.of(slm)).cpu().numpy()
    ref = oracle_front(w)
    sc = Scene(ref["mean"], ref["quat"].astype(np.float32), ref["scale"].astype(np.float32),
               ref["opacity"].astype(np.float32), w.amp)
    want = O.field(sc, slm)
    for l in range(slm.n_lambda):
        assert rel_l2(field[l], want[l]) < 2e-4


def test_front_full_size_sampled():
    # 1M Gaussians at the headline grid: sampled element-wise parity, and the launch time
    slm = SLM(1080, 1920, 8e-6, 8e-6, RGB)
    w = world_scene(9, 1_000_000, slm, n_surfaces=32, volume_frac=0.2)
    wd = world_dev(w)
    cam = camera(w)
    g, valid = gws.holographics(wd, cam, w.holo, compact=False)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(5):
        gws.holographics(wd, cam, w.holo, compact=False)
    e1.record()
    e1.synchronize()
    print(f"front end, 1M Gaussians: {e0.elapsed_time(e1) / 5:.3f} ms per call (incl. allocation)")
    idx = np.random.default_rng(0).choice(w.n, 4000, replace=False)
    sub = world_scene(9, 1, slm)
    sub.mean, sub.quat, sub.scale, sub.sh = w.mean[idx], w.quat[idx], w.scale[idx], w.sh[idx]
    sub.view, sub.holo, sub.fx, sub.fy, sub.cx, sub.cy = w.view, w.holo, w.fx, w.fy, w.cx, w.cy
    ref = oracle_front(sub)
    it = torch.as_tensor(idx, device="cuda")
    gs = gws.Gaussians(g.mean[it], g.quat[it], g.scale[it], g.opacity[it], g.amp[it])
    compare(gs, valid[it], ref, extent=1e-2)
