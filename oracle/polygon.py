"""FP64 oracle of the triangle primitive (the supplement's section on polygon-based methods).

TEST INFRASTRUCTURE ONLY (tests, smoke check, CPU baseline of the benchmark): the product
path never imports this module.

* Canonical triangle: the indicator of P = {(0,0), (1,0), (1,1)}; its spectrum in this code's
  convention (ordinary frequency, e^{-j 2 pi nu . x}) is the supplement's piecewise closed form
  (the integral of e^{j k . x} over P) at k = -2 pi nu, case by case (`canonical_piecewise`).
  The case k_x = -k_y is taken as the limit of the general case, (1 - e^{-j k_y}) / k_y^2 - j / k_y
  (what the integral gives; the printed case has e^{+j k_y}).  The printed form cancels
  catastrophically next to its singular lines, so the spectra use `canonical`, the same integral
  through divided differences, pinned to the printed form and to quadrature.
* A triangle with vertices v1, v2, v3 in hologram space is the canonical one mapped by an
  in-plane rotation R (r1 along v2 - v1, r3 the normal (v2 - v1) x (v3 - v1), r2 = r3 x r1),
  a 2D affine map and the translation mu = v1: x_o = R^T (x - v1) has the vertices V_o =
  [[|v2 - v1|, r1 . (v3 - v1)], [0, r2 . (v3 - v1)]] (columns: vertices 2 and 3), and A V_o = P
  = [[1, 1], [0, 1]] maps them to the canonical ones (x_c = A x_o).
* Spectrum (Eq. 10 with the canonical Gaussian replaced by the canonical triangle; the affine
  theorem of Eq. 8 for x_c = A x_o gives the factor |det A|^-1 and the argument A^-T k_o):
      u_hat(f) = c o |r3 . f| / f_z |det V_o| T_hat(A^-T (r1 . d, r2 . d)) e^{-j 2 pi f . v1},
  d = f - f_r (the reference wave of Sec. 4.1 on axis), summed over triangles as in Eq. 12.
"""
from __future__ import annotations

import numpy as np

from . import oracle as O


def canonical_piecewise(nu_x, nu_y):
    """T_hat(nu) = int_P e^{-j 2 pi nu . x} dx by the supplement's case analysis (k = -2 pi nu)."""
    kx = -2.0 * np.pi * np.asarray(nu_x, dtype=np.float64)
    ky = -2.0 * np.pi * np.asarray(nu_y, dtype=np.float64)
    kx, ky = np.broadcast_arrays(kx, ky)
    out = np.empty(kx.shape, dtype=np.complex128)
    with np.errstate(divide="ignore", invalid="ignore"):
        c0 = (kx == 0) & (ky == 0)
        c1 = (kx == 0) & (ky != 0)
        c2 = (kx != 0) & (ky == 0)
        c3 = (kx == -ky) & (ky != 0) & ~c1 & ~c2
        c4 = ~(c0 | c1 | c2 | c3)
        out[c0] = 0.5
        out[c1] = (1 - np.exp(1j * ky[c1])) / ky[c1] ** 2 + 1j / ky[c1]
        out[c2] = (np.exp(1j * kx[c2]) - 1) / kx[c2] ** 2 - 1j * np.exp(1j * kx[c2]) / kx[c2]
        out[c3] = (1 - np.exp(-1j * ky[c3])) / ky[c3] ** 2 - 1j / ky[c3]
        a, b = kx[c4], ky[c4]
        out[c4] = (np.exp(1j * a) - 1) / (a * b) + (1 - np.exp(1j * (a + b))) / (b * (a + b))
    return out


def canonical(nu_x, nu_y):
    """T_hat(nu), stable everywhere: the integral of e^{l(x)} over a triangle with l linear is
    2 area times the second divided difference of exp at l's vertex values, so with area 1/2
    T_hat(nu) = exp[z0, z1, z2], z = -j 2 pi (0, nu_x, nu_x + nu_y) (the phases at (0,0), (1,0),
    (1,1)).  Spread of the nodes above 0.1: (E[z1,z2] - E[z0,z1]) / (z2 - z0) with z0, z2 the
    extreme nodes and E[p,q] = e^{(p+q)/2} sinh((q-p)/2) / ((q-p)/2); below: the Taylor series
    e^{zbar} sum_k h_k(w) / (k+2)!, w = z - zbar, h_k the complete homogeneous polynomials."""
    a = 2.0 * np.pi * np.asarray(nu_x, dtype=np.float64)
    b = 2.0 * np.pi * np.asarray(nu_y, dtype=np.float64)
    a, b = np.broadcast_arrays(a, b)
    th = np.stack([np.zeros_like(a), -a, -(a + b)])  # z = j th
    th = np.sort(th, axis=0)
    t0, t1, t2 = th[0], th[1], th[2]
    spread = t2 - t0

    def E(p, q):  # first divided difference of exp at j p, j q
        h = 0.5 * (q - p)
        return np.exp(0.5j * (p + q)) * np.sinc(h / np.pi)

    out = np.empty(a.shape, dtype=np.complex128)
    big = spread > 0.1
    with np.errstate(divide="ignore", invalid="ignore"):
        out[big] = ((E(t1, t2) - E(t0, t1)) / (1j * spread))[big]
    tb = (t0 + t1 + t2) / 3.0
    w = [1j * (t - tb) for t in (t0, t1, t2)]
    # h_k(w0, w1, w2) by h_k = sum_m h_m(w0, w1) w2^(k-m), h_m(w0, w1) = sum_i w0^i w1^(m-i)
    series = np.zeros(a.shape, dtype=np.complex128)
    fact = 2.0
    for k in range(14):
        hk = np.zeros(a.shape, dtype=np.complex128)
        for m in range(k + 1):
            h2 = sum(w[0] ** i * w[1] ** (m - i) for i in range(m + 1))
            hk = hk + h2 * w[2] ** (k - m)
        series = series + hk / fact
        fact *= (k + 3)
    out[~big] = (np.exp(1j * tb) * series)[~big]
    return out


def frame(v):
    """(R [n,3,3] columns r1, r2, r3; V_o [n,2,2]; A [n,2,2]) of triangles v [n,3,3] (rows v1, v2, v3)."""
    v = np.asarray(v, dtype=np.float64)
    e2, e3 = v[:, 1] - v[:, 0], v[:, 2] - v[:, 0]
    r1 = e2 / np.linalg.norm(e2, axis=1, keepdims=True)
    nrm = np.cross(e2, e3)
    r3 = nrm / np.linalg.norm(nrm, axis=1, keepdims=True)
    r2 = np.cross(r3, r1)
    R = np.stack([r1, r2, r3], axis=2)
    Vo = np.zeros((v.shape[0], 2, 2))
    Vo[:, 0, 0] = np.sum(r1 * e2, axis=1)
    Vo[:, 0, 1] = np.sum(r1 * e3, axis=1)
    Vo[:, 1, 1] = np.sum(r2 * e3, axis=1)
    A = np.array([[1.0, 1.0], [0.0, 1.0]])[None] @ np.linalg.inv(Vo)
    return R, Vo, A


def _at(vertices, opacity, amp, l, lam, FX, FY, phase_match):
    """Sum over triangles of their spectra at the frequencies (FX, FY) (any shape), wavelength l."""
    R, Vo, A = frame(vertices)
    AinvT = np.transpose(np.linalg.inv(A), (0, 2, 1))
    detVo = np.abs(np.linalg.det(Vo))
    k2 = 1.0 / lam ** 2
    rho2 = FX ** 2 + FY ** 2
    prop = rho2 < k2
    FZ = np.sqrt(np.where(prop, k2 - rho2, 0.0))
    DZ = FZ - 1.0 / lam
    out = np.zeros(FX.shape, dtype=np.complex128)
    for i in range(vertices.shape[0]):
        r1, r2, r3 = R[i, :, 0], R[i, :, 1], R[i, :, 2]
        do = np.stack([r1[0] * FX + r1[1] * FY + r1[2] * DZ, r2[0] * FX + r2[1] * FY + r2[2] * DZ])
        nu = np.tensordot(AinvT[i], do, axes=(1, 0))
        jac = np.abs(r3[0] * FX + r3[1] * FY + r3[2] * FZ) / np.where(prop, FZ, 1.0)
        v1 = vertices[i, 0]
        ph = -2.0 * np.pi * (FX * v1[0] + FY * v1[1] + FZ * v1[2])
        if phase_match:
            ph = ph + 2.0 * np.pi * v1[2] / lam
        t = float(opacity[i]) * float(amp[i, l]) * jac * detVo[i] * canonical(nu[0], nu[1]) * np.exp(1j * ph)
        out += np.where(prop, t, 0.0)
    return out


def spectrum(vertices, opacity, amp, slm, phase_match=False):
    """u_hat_SLM(f), complex128 [n_lambda][H][W], of triangles (vertices [n,3,3], rows v1, v2, v3)."""
    vertices = np.asarray(vertices, dtype=np.float64)
    H, W = slm.H, slm.W
    fx = (np.arange(W) - W // 2) / (W * slm.pitch_x)
    fy = (np.arange(H) - H // 2) / (H * slm.pitch_y)
    FX, FY = np.meshgrid(fx, fy)
    out = np.zeros((slm.n_lambda, H, W), dtype=np.complex128)
    for l, lam in enumerate(slm.wavelengths):
        out[l] = _at(vertices, opacity, amp, l, lam, FX, FY, phase_match)
    return out


def spectrum_at(vertices, opacity, amp, slm, l, rows, cols, phase_match=False):
    """u_hat_SLM at grid samples (rows, cols) of wavelength index l."""
    vertices = np.asarray(vertices, dtype=np.float64)
    FX = (np.asarray(cols) - slm.W // 2) / (slm.W * slm.pitch_x)
    FY = (np.asarray(rows) - slm.H // 2) / (slm.H * slm.pitch_y)
    return _at(vertices, opacity, amp, l, slm.wavelengths[l], FX.astype(np.float64), FY.astype(np.float64),
               phase_match)


def field(vertices, opacity, amp, slm, phase_match=False):
    """u_SLM: the centred inverse DFT (Eq. 3) of `spectrum`."""
    return O.idft(spectrum(vertices, opacity, amp, slm, phase_match), slm.pitch_x, slm.pitch_y)
