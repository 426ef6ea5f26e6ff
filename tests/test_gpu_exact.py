"""GPU parity of exact alpha wave blending (Algorithm S2; blend GWS_BLEND_EXACT) against the
oracle's FP64 restatement of the algorithm (direct DFTs).  Bar: the mixed path's 2e-4 rel-L2."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2505_06582_gb300 import gws
from paper_2505_06582_gb300.scenes import SLM, surface_scene, uniform_scene
from tests.helpers import make_scene, rel_l2

pytestmark = pytest.mark.gpu
TOL = 2e-4


def dev(sc):
    return gws.Gaussians.from_scene(sc, "cuda")


@pytest.mark.parametrize("batch", [0, 3])
@pytest.mark.parametrize("domain", [gws.DOMAIN_SPECTRUM, gws.DOMAIN_FIELD], ids=["spectrum", "field"])
def test_exact_matches_oracle(batch, domain):
    slm = SLM(48, 64, 8e-6, 8e-6, (638e-9, 450e-9))
    sc = surface_scene(70, 24, slm, n_surfaces=2, scale_median_px=3.0)
    ref = O.exact_awb(sc, slm)
    if domain == gws.DOMAIN_FIELD:
        ref = O.idft(ref, slm.pitch_x, slm.pitch_y)
    got = gws.forward(dev(sc), slm, blend=gws.BLEND_EXACT, domain=domain, exact_batch=batch).cpu().numpy()
    for l in range(2):
        assert rel_l2(got[l], ref[l]) < TOL
    # occlusion matters in this scene: exact differs from the order-invariant sum
    assert rel_l2(O.spectrum(sc, slm)[0], O.exact_awb(sc, slm)[0]) > 1e-3


def test_exact_binarized_disks():
    slm = SLM(64, 64, 8e-6, 8e-6, (520e-9,))
    sc = uniform_scene(71, 16, slm, scale_median_px=4.0)
    ref = O.exact_awb(sc, slm, binarize=0.3)
    got = gws.forward(dev(sc), slm, blend=gws.BLEND_EXACT, domain=gws.DOMAIN_SPECTRUM, t_binarize=0.3).cpu().numpy()
    # FP32 vs FP64 decisions at the disk edge (alpha = 0.3) may differ on a few pixels
    assert rel_l2(got, ref) < 2e-3


def test_exact_without_occlusion_equals_the_order_invariant_forward():
    slm = SLM(56, 72, 8e-6, 8e-6, (638e-9, 520e-9, 450e-9))
    sc = surface_scene(72, 30, slm, n_surfaces=3)
    sc.opacity[:] = 0.5 / 255
    g = dev(sc)
    ex = gws.forward(g, slm, blend=gws.BLEND_EXACT, domain=gws.DOMAIN_SPECTRUM).cpu().numpy()
    oit = gws.forward(g, slm, domain=gws.DOMAIN_SPECTRUM).cpu().numpy()
    assert rel_l2(ex, oit) < 2e-5


def test_exact_occluded_rear_is_hidden_by_a_binarized_disk():
    slm = SLM(80, 80, 8e-6, 8e-6, (520e-9,))
    front = make_scene([[0, 0, 2e-3]], [[1, 0, 0, 0]], [[12 * 8e-6, 12 * 8e-6]], [1.0], [[0.6]])
    rear = make_scene([[8e-6, 0, 5e-3]], [[1, 0, 0, 0]], [[2.5 * 8e-6, 2.5 * 8e-6]], [0.9], [[0.8]])
    both = rear.concat(front)
    got = gws.forward(dev(both), slm, blend=gws.BLEND_EXACT, domain=gws.DOMAIN_SPECTRUM, t_binarize=0.05)
    only = gws.forward(dev(front), slm, blend=gws.BLEND_EXACT, domain=gws.DOMAIN_SPECTRUM, t_binarize=0.05)
    assert rel_l2(got.cpu().numpy(), only.cpu().numpy()) < 1e-5


def test_exact_rejects_unsupported_combinations():
    slm = SLM(16, 16, 8e-6, 8e-6, (520e-9,))
    sc = uniform_scene(73, 3, slm)
    with pytest.raises(gws.GwsError) as e:
        gws.forward(dev(sc), slm, blend=gws.BLEND_EXACT, prec=gws.PREC_FP64)
    assert e.value.code == 6
    with pytest.raises(gws.GwsError) as e:
        gws.forward_batched([dev(sc)], slm, blend=gws.BLEND_EXACT)
    assert e.value.code == 6


@pytest.mark.parametrize("H,W", [(50, 64), (45, 61)], ids=["even_origin_sign", "odd"])
def test_exact_grid_parities(H, W):
    # 50 x 64: H/2 + W/2 odd, so the folded modulation constant is negative; 45 x 61: odd sizes,
    # where the explicit modulation passes run
    slm = SLM(H, W, 8e-6, 8e-6, (520e-9,))
    sc = surface_scene(71, 16, slm, n_surfaces=2, scale_median_px=3.0)
    ref = O.idft(O.exact_awb(sc, slm), slm.pitch_x, slm.pitch_y)
    got = gws.forward(dev(sc), slm, blend=gws.BLEND_EXACT, exact_batch=5).cpu().numpy()
    assert rel_l2(got[0], ref[0]) < TOL
