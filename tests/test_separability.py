"""The premise of a tensor-core recast of the splat (a batched complex GEMM over (Gaussian x f_x)
and (Gaussian x f_y)): each Gaussian's spectrum without its lateral ramp, A_i(f) e^{-j 2 pi f_z mu_z},
would have to be (close to) separable on the frequency grid.  On the headline Gaussians (surface
scenes, 8 um pitch) it is not: the best rank-1 approximation misses the mixed path's 2e-4 bar by
orders of magnitude and a rank of several is needed, so the recast is not adopted.
"""
import numpy as np

import oracle as O
from paper_2505_06582_gb300.scenes import SLM, surface_scene


def test_headline_gaussian_spectra_are_not_separable():
    slm = SLM(135, 240, 8e-6, 8e-6, (520e-9,))  # the headline frequency extent, coarser steps
    sc = surface_scene(1, 2000, slm, n_surfaces=32)
    idx = np.random.default_rng(0).choice(sc.n, 40, replace=False)
    err1, ranks = [], []
    for i in idx:
        t, _ = O.single_terms(np.array([0.0, 0.0, sc.mean[i, 2]]), sc.quat[i].astype(np.float64),
                              sc.scale[i].astype(np.float64), 520e-9, slm.H, slm.W, slm.pitch_x, slm.pitch_y)
        s = np.linalg.svd(t, compute_uv=False)
        tail = np.sqrt(np.cumsum((s ** 2)[::-1])[::-1]) / np.sqrt(np.sum(s ** 2))  # tail[r]: rank-r error
        err1.append(tail[1])
        ranks.append(int(np.argmax(tail < 2e-4)) if np.any(tail < 2e-4) else len(s))
    assert np.median(err1) > 100 * 2e-4
    assert np.median(ranks) >= 3
