"""Pins of the triangle-primitive oracle (oracle/polygon.py; the supplement's polygon section).

* The canonical spectrum against Gauss-Legendre quadrature of the defining integral over the
  reference triangle (Duffy map), at generic frequencies, on each special case of the piecewise
  form, and next to the singular lines.
* An untilted triangle's hologram-space spectrum against direct quadrature of the 2D Fourier
  integral of its indicator (pins the affine map, its determinant and the translation).
* Relabelling the vertices (cyclic shifts and reversed orientation) leaves a tilted, displaced
  triangle's spectrum unchanged.
"""
import numpy as np
import pytest

from oracle import polygon as PG
from paper_2505_06582_gb300.scenes import SLM
from tests.helpers import rel_l2


def _gl_triangle(nu_x, nu_y, n=48):
    """int_{0 <= y <= x <= 1} e^{-j 2 pi (nu_x x + nu_y y)} dx dy by x = u, y = u v (dA = u du dv)."""
    g, w = np.polynomial.legendre.leggauss(n)
    u, wu = 0.5 * (g + 1), 0.5 * w
    U, V = np.meshgrid(u, u, indexing="ij")
    WW = np.outer(wu, wu)
    x, y = U, U * V
    return np.sum(WW * U * np.exp(-2j * np.pi * (nu_x * x + nu_y * y)))


def test_canonical_spectrum_against_quadrature():
    # the printed piecewise form (with the k_x = -k_y case taken as the integral's limit) and the
    # divided-difference form against quadrature; next to the singular lines only the latter
    rng = np.random.default_rng(0)
    pts = [(0.0, 0.0), (0.0, 1.3), (-0.7, 0.0), (0.9, -0.9), (-1.7, 1.7), (0.0, -2.2)]
    pts += [tuple(v) for v in rng.uniform(-2.5, 2.5, (30, 2))]
    pts += [(1.1, 1e-4), (1e-4, -0.8), (0.6, -0.6 + 1e-4), (2.0, 3e-3)]
    for nx, ny in pts:
        want = _gl_triangle(nx, ny)
        got = PG.canonical_piecewise(np.array(nx), np.array(ny))
        assert abs(got - want) < 1e-8, (nx, ny, got, want)
        assert abs(PG.canonical(np.array(nx), np.array(ny)) - want) < 1e-12, (nx, ny)
    for nx, ny in [(1e-11, 3e-12), (-2e-9, 1e-9), (0.3, 1e-13), (1e-12, -0.5), (0.02, -0.0199999)]:
        assert abs(PG.canonical(np.array(nx), np.array(ny)) - _gl_triangle(nx, ny)) < 1e-12, (nx, ny)
    # the spread threshold between the two branches leaves no step
    eps = 1e-9
    s = 0.1 / (2 * np.pi)
    lo = PG.canonical(np.array(s - eps), np.array(0.0))
    hi = PG.canonical(np.array(s + eps), np.array(0.0))
    assert abs(hi - lo) < 1e-8


def _triangle_ft(v, fx, fy, n=64):
    """2D Fourier integral of the indicator of the planar triangle v (z ignored) at (fx, fy)."""
    g, w = np.polynomial.legendre.leggauss(n)
    u, wu = 0.5 * (g + 1), 0.5 * w
    U, V = np.meshgrid(u, u, indexing="ij")
    WW = np.outer(wu, wu)
    # x = v1 + u (v2 - v1) + u s (v3 - v2): the Duffy map of the triangle, |J| = u |(v2-v1) x (v3-v2)|
    e1, e2 = v[1, :2] - v[0, :2], v[2, :2] - v[1, :2]
    jac = abs(e1[0] * e2[1] - e1[1] * e2[0])
    X = v[0, 0] + U * e1[0] + U * V * e2[0]
    Y = v[0, 1] + U * e1[1] + U * V * e2[1]
    out = np.empty(fx.shape, dtype=np.complex128)
    for idx in np.ndindex(fx.shape):
        out[idx] = np.sum(WW * U * jac * np.exp(-2j * np.pi * (fx[idx] * X + fy[idx] * Y)))
    return out


def test_untilted_triangle_is_the_fourier_integral_of_its_indicator():
    slm = SLM(12, 14, 8e-6, 8e-6, (520e-9,))
    p = 8e-6
    v = np.array([[[3 * p, -2 * p, 0.0], [9 * p, 1 * p, 0.0], [1 * p, 6 * p, 0.0]]])
    spec = PG.spectrum(v, np.ones(1), np.ones((1, 1)), slm)[0]
    fx = (np.arange(slm.W) - slm.W // 2) / (slm.W * p)
    fy = (np.arange(slm.H) - slm.H // 2) / (slm.H * p)
    FX, FY = np.meshgrid(fx, fy)
    want = _triangle_ft(v[0], FX, FY)
    assert rel_l2(spec, want) < 1e-9


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_vertex_relabelling(seed):
    # The shape factor sees d = f - f_r and the ramp f, so the first vertex fixes the phase of the
    # reference wave's carrier: relabelling multiplies a triangle's spectrum by exp(-j 2 pi dz / lambda)
    # (dz the new first vertex's depth minus the old one's), and with phase matching (carrier
    # referenced to the global reference wave) the spectrum does not depend on the labelling.
    rng = np.random.default_rng(seed)
    slm = SLM(16, 20, 8e-6, 8e-6, (638e-9, 450e-9))
    c = np.array([rng.uniform(-40e-6, 40e-6), rng.uniform(-40e-6, 40e-6), rng.uniform(1e-3, 3e-3)])
    v = c + rng.normal(size=(3, 3)) * np.array([30e-6, 30e-6, 10e-6])
    amp = np.array([[0.7, 0.4]])
    ref = PG.spectrum(v[None], np.array([0.8]), amp, slm)
    ref_pm = PG.spectrum(v[None], np.array([0.8]), amp, slm, phase_match=True)
    for perm in ([1, 2, 0], [2, 0, 1], [0, 2, 1], [2, 1, 0]):
        got = PG.spectrum(v[perm][None], np.array([0.8]), amp, slm)
        got_pm = PG.spectrum(v[perm][None], np.array([0.8]), amp, slm, phase_match=True)
        dz = v[perm][0, 2] - v[0, 2]
        for l, lam in enumerate(slm.wavelengths):
            assert rel_l2(got_pm[l], ref_pm[l]) < 1e-10, perm
            assert rel_l2(got[l], ref[l] * np.exp(-2j * np.pi * dz / lam)) < 1e-10, perm


@pytest.mark.parametrize("seed", [4, 5])
def test_tilted_triangle_remap_and_jacobian(seed):
    # u_hat(f) = |det d(k_o)/d(f_xy)| (finite differences of the remap (f_x, f_y) -> (r1.d, r2.d))
    #            x the Fourier integral of the indicator in the triangle's own plane at k_o
    #            x e^{-j 2 pi f . v1}: independent of the closed form, the affine map and the
    #            Jacobian reading |r3 . f| / f_z
    rng = np.random.default_rng(seed)
    lam = 520e-9
    slm = SLM(10, 12, 4e-6, 4e-6, (lam,))
    c = np.array([rng.uniform(-10e-6, 10e-6), rng.uniform(-10e-6, 10e-6), 1.5e-3])
    v = c + rng.normal(size=(3, 3)) * np.array([8e-6, 8e-6, 6e-6])
    spec = PG.spectrum(v[None], np.ones(1), np.ones((1, 1)), slm)[0]
    R, Vo, _ = PG.frame(v[None])
    r1, r2 = R[0, :, 0], R[0, :, 1]
    tri_o = np.array([[0.0, 0.0, 0.0], [Vo[0, 0, 0], 0.0, 0.0], [Vo[0, 0, 1], Vo[0, 1, 1], 0.0]])

    def k_o(fx, fy):
        fz = np.sqrt(1 / lam ** 2 - fx * fx - fy * fy)
        d = np.array([fx, fy, fz - 1 / lam])
        return np.array([r1 @ d, r2 @ d]), fz

    for (r, cc) in [(3, 4), (5, 6), (8, 1), (0, 11), (7, 9)]:
        fx = (cc - slm.W // 2) / (slm.W * slm.pitch_x)
        fy = (r - slm.H // 2) / (slm.H * slm.pitch_y)
        h = 1.0
        kx1, _ = k_o(fx + h, fy)
        kx0, _ = k_o(fx - h, fy)
        ky1, _ = k_o(fx, fy + h)
        ky0, _ = k_o(fx, fy - h)
        jac = abs(np.linalg.det(np.stack([(kx1 - kx0) / (2 * h), (ky1 - ky0) / (2 * h)], axis=1)))
        ko, fz = k_o(fx, fy)
        ft = _triangle_ft(tri_o, np.array([ko[0]]), np.array([ko[1]]))[0]
        want = jac * ft * np.exp(-2j * np.pi * (fx * v[0, 0] + fy * v[0, 1] + fz * v[0, 2]))
        assert abs(spec[r, cc] - want) < 1e-7 * abs(Vo[0, 0, 0] * Vo[0, 1, 1]), (r, cc, spec[r, cc], want)
