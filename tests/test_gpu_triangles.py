"""GPU parity of the triangle primitive (gws_forward_triangles, the supplement's polygon section)
against the FP64 oracle (oracle/polygon.py): relative L2 per wavelength <= 2e-4 for the field and
the spectrum, phase matching, relabelling invariance under phase matching, degenerate and
non-finite triangles recorded in the status word, empty input, and the dense cost at the
Tab. 3 shape."""
import numpy as np
import pytest
import torch

from oracle import polygon as PG
from paper_2505_06582_gb300 import gws
from paper_2505_06582_gb300.scenes import SLM, triangle_scene
from tests.helpers import rel_l2

pytestmark = pytest.mark.gpu

TOL = 2e-4


def dev(verts, opa, amp):
    t = lambda a, dt: torch.as_tensor(np.ascontiguousarray(a), dtype=dt, device="cuda")
    return t(verts, torch.float64), t(opa, torch.float32), t(amp, torch.float32)


@pytest.mark.parametrize("slm,n,seed", [(SLM(48, 64, 8e-6, 8e-6, (638e-9, 520e-9)), 20, 1),
                                        (SLM(37, 53, 8e-6, 6e-6, (450e-9,)), 15, 2),
                                        (SLM(64, 64, 4e-6, 4e-6, (520e-9,)), 12, 3)])
@pytest.mark.parametrize("domain", [gws.DOMAIN_FIELD, gws.DOMAIN_SPECTRUM])
def test_triangles_match_oracle(slm, n, seed, domain):
    verts, opa, amp = triangle_scene(seed, n, slm, size_px=4.0)
    got = gws.forward_triangles(*dev(verts, opa, amp), gws.Slm.of(slm), domain=domain).cpu().numpy()
    want = (PG.field if domain == gws.DOMAIN_FIELD else PG.spectrum)(verts, opa, amp, slm)
    for l in range(slm.n_lambda):
        assert rel_l2(got[l], want[l]) < TOL, (l, rel_l2(got[l], want[l]))


def test_triangles_phase_match_and_relabelling():
    slm = SLM(40, 48, 8e-6, 8e-6, (520e-9, 638e-9))
    verts, opa, amp = triangle_scene(4, 10, slm, size_px=5.0)
    S = gws.Slm.of(slm)
    got = gws.forward_triangles(*dev(verts, opa, amp), S, phase_match=True).cpu().numpy()
    want = PG.field(verts, opa, amp, slm, phase_match=True)
    for l in range(slm.n_lambda):
        assert rel_l2(got[l], want[l]) < TOL
    perm = gws.forward_triangles(*dev(verts[:, [2, 0, 1]], opa, amp), S, phase_match=True).cpu().numpy()
    for l in range(slm.n_lambda):
        assert rel_l2(perm[l], got[l]) < 1e-5


def test_triangles_degenerate_nonfinite_and_empty():
    slm = SLM(32, 32, 8e-6, 8e-6, (520e-9,))
    S = gws.Slm.of(slm)
    verts, opa, amp = triangle_scene(5, 6, slm)
    ref = PG.field(verts[1:], opa[1:], amp[1:], slm)
    bad = verts.copy()
    bad[0, 2] = bad[0, 0] + 0.5 * (bad[0, 1] - bad[0, 0])  # collinear: zero area
    opts = dict(workspace=torch.empty(1 << 24, dtype=torch.uint8, device="cuda"))
    got = gws.forward_triangles(*dev(bad, opa, amp), S, **opts).cpu().numpy()
    assert rel_l2(got[0], ref[0]) < TOL  # the degenerate one contributes nothing
    st = gws.load().gws_get_device_status(__import__("ctypes").byref(_opts_with_ws(opts["workspace"])))
    assert st == 1  # GWS_ERR_INVALID_ARG: a bad value was recorded
    nanv = verts.copy()
    nanv[0, 1, 0] = np.nan
    gws.forward_triangles(*dev(nanv, opa, amp), S, **opts)
    st = gws.load().gws_get_device_status(__import__("ctypes").byref(_opts_with_ws(opts["workspace"])))
    assert st == 4  # GWS_ERR_NONFINITE
    z = gws.forward_triangles(*dev(np.zeros((0, 3, 3)), np.zeros(0), np.zeros((0, 1))), S)
    assert torch.count_nonzero(z) == 0


def _opts_with_ws(ws):
    o = gws.make_opts()
    o.workspace = __import__("ctypes").c_void_p(ws.data_ptr())
    o.workspace_bytes = ws.numel()
    return o


def test_triangles_tab3_time():
    # 15k triangles at 1024 x 1280 (the Tab. 3 shape), dense: sampled parity and the launch time
    slm = SLM(1024, 1280, 8e-6, 8e-6, (520e-9,))
    verts, opa, amp = triangle_scene(6, 15_000, slm, size_px=3.0)
    S = gws.Slm.of(slm)
    d = dev(verts, opa, amp)
    out = gws.forward_triangles(*d, S, domain=gws.DOMAIN_SPECTRUM)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    gws.forward_triangles(*d, S, out=out, domain=gws.DOMAIN_SPECTRUM)
    e1.record()
    e1.synchronize()
    ms = e0.elapsed_time(e1)
    print(f"triangles, 15k @ 1024x1280 (dense, spectrum): {ms:.1f} ms, "
          f"{15_000 * 1024 * 1280 / (ms * 1e-3):.3g} pairs/s")
    sub = np.random.default_rng(0).choice(15_000, 200, replace=False)
    # linearity: the spectrum of a subset equals the sum over it (oracle on the subset)
    part = gws.forward_triangles(*dev(verts[sub], opa[sub], amp[sub]), S, domain=gws.DOMAIN_SPECTRUM).cpu().numpy()
    rows = np.random.default_rng(1).integers(0, 1024, 256)
    cols = np.random.default_rng(2).integers(0, 1280, 256)
    want = PG.spectrum_at(verts[sub], opa[sub], amp[sub], slm, 0, rows, cols)
    assert rel_l2(part[0][rows, cols], want) < TOL
