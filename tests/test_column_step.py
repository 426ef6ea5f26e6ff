"""Host-side checks of the forward splat's column step (splat_record_step in
csrc/gws_splat.cu): the facts its guard rests on, in FP64 numpy.

A thread owns 8 consecutive columns of one row (columns c0 + 0..7, c0 a multiple of 8 inside
64-column tiles); its odd packs hold columns c0 + {1, 3, 5, 7}, each one column right of an even
pack's c0 + {0, 2, 4, 6}.  Per record the odd pixel's phase is the even one's plus
beta = t_x dfx + t_z sbar (sbar: the thread's mean step of f_z) plus t_z dl, dl the pixel's
residual step, and e^{j t_z dl} is taken to first order.  The kernel's comments state a bound on
max |dl| for the 1920- and 3840-column grids and the depth range over which the first-order
residual stays within its 2e-3 rad threshold; these tests recompute both, and check the
rotation identity and its error against the exact phase factor."""
import math
import os
import re

import numpy as np
import pytest

SRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "paper_2505_06582_gb300", "csrc",
                   "gws_splat.cu")
RGB = (638e-9, 520e-9, 450e-9)


def _step_eps():
    return float(re.search(r"constexpr float kStepEps = ([0-9.e-]+)f;", open(SRC).read()).group(1))


def _residuals(H, W, pitch, lam):
    """Per thread: sbar and the residual steps dl of its four even -> odd pairs (valid pixels)."""
    fx = (np.arange(W) - W // 2) / (W * pitch)
    fy = (np.arange(H) - H // 2) / (H * pitch)
    fz = np.sqrt(1.0 / lam**2 - fx[None, :] ** 2 - fy[:, None] ** 2)  # no evanescent pixels on these grids
    Wt = (W // 8) * 8
    z = fz[:, :Wt].reshape(H, Wt // 8, 8)
    step = z[:, :, 1::2] - z[:, :, 0::2]
    sbar = step.mean(axis=-1, keepdims=True)
    return sbar, step - sbar


@pytest.mark.parametrize("H,W,pitch", [(1080, 1920, 8e-6), (2160, 3840, 3.74e-6)])
def test_residual_step_bound_on_the_large_grids(H, W, pitch):
    eps = _step_eps()
    for lam in RGB:
        _, dl = _residuals(H, W, pitch, lam)
        dmax = np.abs(dl).max()
        assert dmax <= 0.0095, (lam, dmax)
        # every record with |mu_z| <= 33 mm takes the column step: |t_z| max|dl| <= kStepEps
        assert 2 * math.pi * 33e-3 * dmax <= eps, (lam, dmax)


def test_first_order_rotation_matches_the_exact_phase_factor():
    """cis(phi_odd) against cis(phi_even) cis(beta) (1 + j t_z dl) at the kernel's worst residual
    phase: the error is (t_z dl)^2 / 2 + O(.^3) <= 2e-6 at the threshold."""
    eps = _step_eps()
    rng = np.random.default_rng(3)
    phi = rng.uniform(-math.pi, math.pi, 10000)
    beta = rng.uniform(-math.pi, math.pi, 10000)
    e = rng.uniform(-eps, eps, 10000)
    exact = np.exp(1j * (phi + beta + e))
    q = np.exp(1j * beta)
    rot = (q.real - e * q.imag) + 1j * (q.imag + e * q.real)  # Re / Im of e^{j beta} (1 + j e), as in the kernel
    approx = np.exp(1j * phi) * rot
    err = np.abs(approx - exact)
    assert np.all(err <= 0.5 * e**2 * (1 + e**2) + 1e-15)
    assert err.max() <= 2.0e-6


def test_the_odd_pixel_gets_the_exact_phase_when_its_neighbour_has_none():
    """An even pixel without amplitude takes f_z - f0_z = its right neighbour's minus sbar, so the
    neighbour's residual is 0 and the carried phase is the neighbour's own (exactly, in FP64)."""
    rng = np.random.default_rng(5)
    tx, tz, tr = rng.normal(size=3) * 100
    dfx, sbar, dz_odd, ddx_even = 65.1, 2.4, 37.0, -4 * 65.1
    dz_even = dz_odd - sbar  # the kernel's substitute
    phi_even = tr + tx * ddx_even + tz * dz_even
    beta = tx * dfx + tz * sbar
    dl = 0.0
    phi_odd = phi_even + beta + tz * dl
    assert phi_odd == pytest.approx(tr + tx * (ddx_even + dfx) + tz * dz_odd, rel=0, abs=1e-9)
