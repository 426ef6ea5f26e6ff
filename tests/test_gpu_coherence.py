"""GPU parity of partially coherent GWS (Eq. 14, GWS_BLEND_PARTIAL_COHERENT) against the FP64 oracle
(oracle/coherence.py): one frame per call, relative L2 per wavelength <= 2e-4 (the mixed path's
bar), on coarse (8 um) and fine (1 um, where the angular kernel varies across the grid) pitches,
every batch split, phase matching, determinism and frame independence, argument checks.
"""
import numpy as np
import pytest
import torch

from oracle import coherence as PC
from paper_2505_06582_gb300 import gws
from paper_2505_06582_gb300.scenes import SLM, uniform_scene
from tests.helpers import rel_l2

pytestmark = pytest.mark.gpu

TOL = 2e-4


def run(sc, slm, l, m, seed, frame, **kw):
    g = gws.Gaussians.from_scene(sc, "cuda")
    return gws.forward(g, gws.Slm.of(slm), blend=gws.BLEND_PARTIAL_COHERENT, pc_l=l, pc_m=m, pc_seed=seed,
                       pc_frame=frame, **kw).cpu().numpy()


CASES = [
    (SLM(48, 64, 8e-6, 8e-6, (638e-9, 520e-9)), 8, 0, 0, 1, 0),
    (SLM(48, 64, 8e-6, 8e-6, (520e-9,)), 8, 1, 1, 2, 5),
    (SLM(40, 56, 1e-6, 1e-6, (520e-9, 450e-9)), 6, 1, -1, 3, 1),
    (SLM(40, 56, 1e-6, 1e-6, (638e-9,)), 6, 2, -2, 4, 7),
    (SLM(33, 45, 1.2e-6, 1e-6, (520e-9,)), 5, 3, 0, 9, 2),
    (SLM(50, 64, 8e-6, 8e-6, (520e-9,)), 6, 1, 0, 4, 3),  # H/2 + W/2 odd: the folded constant is negative
]


@pytest.mark.parametrize("slm,n,l,m,seed,frame", CASES)
def test_partial_coherence_matches_oracle(slm, n, l, m, seed, frame):
    zr = (1e-3, 3e-3) if slm.pitch_x > 4e-6 else (20e-6, 80e-6)
    sc = uniform_scene(seed, n, slm, z_range=zr, scale_median_px=3.0)
    got = run(sc, slm, l, m, seed, frame)
    want = PC.field(sc, slm, l, m, seed, frame)
    for k in range(slm.n_lambda):
        assert rel_l2(got[k], want[k]) < TOL, (k, rel_l2(got[k], want[k]))


def test_partial_coherence_batches_and_phase_match():
    slm = SLM(40, 48, 8e-6, 8e-6, (520e-9, 638e-9))
    sc = uniform_scene(12, 9, slm, z_range=(1e-3, 4e-3), scale_median_px=3.0)
    full = run(sc, slm, 1, 0, 5, 3)
    split = run(sc, slm, 1, 0, 5, 3, exact_batch=4)  # batches of 4, 4, 1
    for k in range(slm.n_lambda):
        assert rel_l2(split[k], full[k]) < 1e-5
    got = run(sc, slm, 1, 0, 5, 3, phase_match=True)
    want = PC.field(sc, slm, 1, 0, 5, 3, phase_match=True)
    for k in range(slm.n_lambda):
        assert rel_l2(got[k], want[k]) < TOL


@pytest.mark.parametrize("slm", [SLM(48, 64, 8e-6, 8e-6, (638e-9, 520e-9)), SLM(33, 45, 1.2e-6, 1e-6, (520e-9,))])
def test_partial_coherence_frames_in_one_call(slm):
    # pc_frames = 3 shares each batch's fields among the frames: every frame equals its own call
    zr = (1e-3, 3e-3) if slm.pitch_x > 4e-6 else (20e-6, 80e-6)
    sc = uniform_scene(31, 9, slm, z_range=zr, scale_median_px=3.0)
    kw = dict(blend=gws.BLEND_PARTIAL_COHERENT, pc_l=1, pc_m=1, pc_seed=3, exact_batch=4)
    g = gws.Gaussians.from_scene(sc, "cuda")
    S = gws.Slm.of(slm)
    multi = gws.forward(g, S, pc_frame=2, pc_frames=3, **kw).cpu().numpy()
    assert multi.shape == (3, slm.n_lambda, slm.H, slm.W)
    for f in range(3):
        one = gws.forward(g, S, pc_frame=2 + f, **kw).cpu().numpy()
        for k in range(slm.n_lambda):
            assert rel_l2(multi[f, k], one[k]) < 1e-6, (f, k)
    want = PC.field(sc, slm, 1, 1, 3, 3)
    for k in range(slm.n_lambda):
        assert rel_l2(multi[1, k], want[k]) < TOL


def test_partial_coherence_frames_are_deterministic_and_independent():
    slm = SLM(32, 32, 8e-6, 8e-6, (520e-9,))
    sc = uniform_scene(13, 4, slm, z_range=(1e-3, 2e-3), scale_median_px=3.0)
    a = run(sc, slm, 0, 0, 77, 0)
    b = run(sc, slm, 0, 0, 77, 0)
    c = run(sc, slm, 0, 0, 77, 1)
    d = run(sc, slm, 0, 0, 78, 0)
    assert np.array_equal(a, b)
    assert rel_l2(c, a) > 0.5 and rel_l2(d, a) > 0.5


def test_partial_coherence_empty_and_arguments():
    slm = SLM(16, 16, 8e-6, 8e-6, (520e-9,))
    sc0 = uniform_scene(1, 0, slm)
    assert np.all(run(sc0, slm, 2, 1, 0, 0) == 0)
    # several frames of an empty scene: every frame's slab is cleared (the output is [F, L, H, W])
    g0 = gws.Gaussians.from_scene(sc0, "cuda")
    dirty = torch.full((3, 1, 16, 16), complex(7.0, -3.0), dtype=torch.complex64, device="cuda")
    got = gws.forward(g0, gws.Slm.of(slm), out=dirty, blend=gws.BLEND_PARTIAL_COHERENT, pc_l=1, pc_m=1,
                      pc_frames=3).cpu().numpy()
    assert got.shape == (3, 1, 16, 16) and np.all(got == 0)
    sc = uniform_scene(1, 3, slm)
    g = gws.Gaussians.from_scene(sc, "cuda")
    S = gws.Slm.of(slm)
    for l, m in ((4, 0), (1, 2), (2, -3), (-1, 0)):
        with pytest.raises(gws.GwsError):
            gws.forward(g, S, blend=gws.BLEND_PARTIAL_COHERENT, pc_l=l, pc_m=m)
    cot = torch.zeros((1, 16, 16), dtype=torch.complex64, device="cuda")
    for blend in (gws.BLEND_PARTIAL_COHERENT, gws.BLEND_EXACT):  # both forward-only
        with pytest.raises(gws.GwsError) as e:
            gws.backward(g, S, cot, blend=blend)
        assert e.value.code == 6  # GWS_ERR_UNSUPPORTED


def test_partial_coherence_tab3_frame_time():
    # one frame at the Tab. 3 shape (15k Gaussians, 1024x1280): sampled parity and the time
    from paper_2505_06582_gb300.scenes import config_scene
    sc, slm = config_scene("paper_tab3_1024x1280")
    g = gws.Gaussians.from_scene(sc, "cuda")
    S = gws.Slm.of(slm)
    kw = dict(blend=gws.BLEND_PARTIAL_COHERENT, pc_l=1, pc_m=1, pc_seed=1, pc_frame=0)
    out = gws.forward(g, S, **kw)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    gws.forward(g, S, out=out, **kw)
    e1.record()
    e1.synchronize()
    print(f"partial coherence, 15k Gaussians @ 1024x1280, one frame: {e0.elapsed_time(e1):.1f} ms")
    # four frames in one call share each batch's fields
    multi = gws.forward(g, S, pc_frames=4, **kw)
    torch.cuda.synchronize()
    e0.record()
    gws.forward(g, S, out=multi, pc_frames=4, **kw)
    e1.record()
    e1.synchronize()
    print(f"partial coherence, 15k Gaussians @ 1024x1280, four frames in one call: {e0.elapsed_time(e1) / 4:.1f} ms per frame")
    assert torch.isfinite(torch.view_as_real(multi)).all()
    assert torch.isfinite(torch.view_as_real(out)).all()
    # the frame's energy: with E|kappa|^2 = 1 the mean intensity is close to the coherent field's
    coh = gws.forward(g, S)
    r = (out.abs() ** 2).mean().item() / (coh.abs() ** 2).mean().item()
    assert 0.3 < r < 3.0
