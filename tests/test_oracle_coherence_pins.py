"""Pins of the partially coherent GWS oracle (Eq. 14; oracle/coherence.py).

* SplitMix64 reproduces the published first outputs of the seed-0 stream.
* The coherent limit (kappa = 1) is exactly Eq. 12's order-invariant field.
* Translating a Gaussian by whole pixels translates its frame exactly (the kernel rides with it).
* Monte Carlo over frames: E|kappa|^2 = 1, and the frame-averaged |V(f)|^2 of one Gaussian
  matches the expectation (1 / sum Y^2) sum_f' Y(f')^2 |G(f - f')|^2 computed by a circular
  convolution in frequency (an independent route).
* The phases are uniform on [-pi, pi) and independent across frames.
"""
import numpy as np
import pytest

import oracle as O
from oracle import coherence as PC
from paper_2505_06582_gb300.scenes import SLM, Scene, uniform_scene
from tests.helpers import rel_l2


def test_splitmix64_known_answers():
    z = PC.splitmix64(np.uint64(0), np.arange(1, 4, dtype=np.uint64))
    assert [int(v) for v in z] == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]


def test_phases_uniform_and_frame_independent():
    slm = SLM(64, 96, 8e-6, 8e-6, (520e-9, 450e-9))
    p0 = PC.phases(slm, 7, 0)
    p1 = PC.phases(slm, 7, 1)
    assert p0.min() >= -np.pi and p0.max() < np.pi
    hist, _ = np.histogram(p0, bins=16, range=(-np.pi, np.pi))
    exp = p0.size / 16
    chi2 = np.sum((hist - exp) ** 2 / exp)
    assert chi2 < 45.0  # 15 dof: p ~ 1e-4
    c = np.corrcoef(np.cos(p0).ravel(), np.cos(p1).ravel())[0, 1]
    assert abs(c) < 5.0 / np.sqrt(p0.size)
    assert not np.array_equal(p0[0], p0[1])  # wavelengths draw their own phases


def test_angular_kernel_values():
    # |K| is the named harmonic of the propagation direction; arg K is the drawn phase
    slm = SLM(16, 20, 0.5e-6, 0.6e-6, (520e-9, 638e-9))
    for l in range(slm.n_lambda):
        FX, FY, FZ, prop = PC.frequencies(slm, l)
        lam = slm.wavelengths[l]
        c1 = np.sqrt(3 / (4 * np.pi))
        c2 = np.sqrt(15 / (4 * np.pi))
        for (sl, sm), want in (((1, 1), c1 * np.abs(lam * FX)), ((1, -1), c1 * np.abs(lam * FY)),
                               ((1, 0), c1 * np.abs(lam * FZ)), ((2, -2), c2 * np.abs(lam * lam * FX * FY))):
            K, _ = PC.angular_kernel(slm, sl, sm, 3, 4)
            assert np.allclose(np.abs(K[l]), np.where(prop, want, 0.0), atol=1e-14)
        K, _ = PC.angular_kernel(slm, 1, 0, 3, 4)  # Y_1^0 > 0 on the propagating grid
        phi = PC.phases(slm, 3, 4)[l]
        d = np.angle(K[l] * np.exp(-1j * phi))
        assert np.all(np.abs(d[prop]) < 1e-12)


@pytest.mark.parametrize("pm", [False, True])
def test_coherent_limit_is_eq12(pm):
    slm = SLM(40, 56, 8e-6, 8e-6, (638e-9, 520e-9))
    sc = uniform_scene(3, 6, slm, z_range=(1e-3, 3e-3), scale_median_px=3.0)
    ones = np.ones((slm.n_lambda, slm.H, slm.W), dtype=np.complex128)
    got = PC.field(sc, slm, 0, 0, 0, 0, phase_match=pm, kappa=ones)
    want = O.field(sc, slm, phase_match=pm)
    for l in range(slm.n_lambda):
        assert rel_l2(got[l], want[l]) < 1e-10  # two direct DFTs and ramps of ~400 cycles in FP64


def test_whole_pixel_translation_moves_the_frame():
    slm = SLM(32, 48, 8e-6, 8e-6, (520e-9,))
    q = np.array([[0.9, 0.1, 0.3, -0.2]], dtype=np.float32)
    q /= np.linalg.norm(q)
    s = np.array([[20e-6, 12e-6]], dtype=np.float32)
    a = Scene(np.zeros((1, 3)), q, s, np.ones(1, np.float32), np.ones((1, 1), np.float32))
    b = Scene(np.array([[3 * 8e-6, -2 * 8e-6, 0.0]]), q, s, np.ones(1, np.float32), np.ones((1, 1), np.float32))
    fa = PC.field(a, slm, 1, -1, 5, 2)
    fb = PC.field(b, slm, 1, -1, 5, 2)
    assert rel_l2(fb, np.roll(fa, shift=(-2, 3), axis=(1, 2))) < 1e-10


def test_kernel_pattern_has_unit_mean_intensity():
    slm = SLM(24, 32, 8e-6, 8e-6, (520e-9,))
    T = 300
    acc = np.zeros((slm.H, slm.W))
    for t in range(T):
        acc += np.abs(PC.kernel_pattern(slm, 1, 1, 11, t)[0]) ** 2
    acc /= T
    assert abs(acc.mean() - 1.0) < 0.02
    assert np.abs(acc - 1.0).max() < 0.4  # per pixel: ~ 1 +- 3 / sqrt(T)


@pytest.mark.parametrize("sh", [(0, 0), (1, 1), (2, -2)])
def test_frame_average_spectrum_matches_the_expectation(sh):
    # tiny pitch so that the angular kernel varies across the grid
    slm = SLM(24, 24, 0.4e-6, 0.4e-6, (520e-9,))
    q = np.array([[1.0, 0, 0, 0]], dtype=np.float32)
    one = Scene(np.zeros((1, 3)), q, np.array([[1.5e-6, 1.0e-6]], np.float32), np.ones(1, np.float32),
                np.ones((1, 1), np.float32))
    T = 400
    avg = np.zeros((slm.H, slm.W))
    for t in range(T):
        avg += np.abs(PC.spectrum(one, slm, sh[0], sh[1], 21, t)[0]) ** 2
    avg /= T
    want = PC.expected_power(one, slm, sh[0], sh[1])[0]
    # Monte-Carlo: relative L2 of the mean over T frames ~ 1 / sqrt(T)
    assert rel_l2(avg, want) < 0.15
    if want.std() > 1e-3 * want.mean():  # l = 0: the expectation is flat, nothing to correlate
        assert np.corrcoef(avg.ravel(), want.ravel())[0, 1] > 0.97
