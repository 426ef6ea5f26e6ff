"""The per-tile spectral footprint bound the splats cull with, checked on CPU in FP64 from its
derivation (truncation of Eq. 10's Gaussian factor at trunc_eps):

  v = (s_u r1.d, s_v r2.d) = M^T f + d_z w,   M = [s_u r1_xy, s_v r2_xy],  w = (s_u r1z, s_v r2z),
  E = 2 pi^2 |v|^2 <= tau = ln(1 / eps)   implies   |M^T f| <= rho_t = sqrt(tau / 2 pi^2) + dzt |w|,

with d = f - f_r, d_z = f_z - 1/lambda and dzt the tile's largest |d_z|, found at the tile's
pixel farthest from f = 0.  The kernels hold the grid-wide ellipse (rho' with the grid's largest
|d_z|, dzmax) in the record and scale it per tile by (rho' / rho_t)^2 = 1 / (1 - (dzmax - dzt) wz)^2,
wz = |w| / rho'.  Every pixel of a tile whose exponent is within the truncation must lie in the
scaled ellipse; the tests sample Gaussians with strong tilts (large |w|) and tiles across the grid."""
import math

import numpy as np
import pytest

TAU = math.log(1.0 / 1e-5)


def _rot(q):
    w, x, y, z = q / np.linalg.norm(q)
    r1 = np.array([1 - 2 * (y * y + z * z), 2 * (x * y + w * z), 2 * (x * z - w * y)])
    r2 = np.array([2 * (x * y - w * z), 1 - 2 * (x * x + z * z), 2 * (y * z + w * x)])
    return r1, r2


def _grid(H, W, p, lam):
    fx = (np.arange(W) - W // 2) / (W * p)
    fy = (np.arange(H) - H // 2) / (H * p)
    FX, FY = np.meshgrid(fx, fy)
    fz = np.sqrt(1.0 / lam**2 - FX**2 - FY**2)
    return FX, FY, fz - 1.0 / lam


def _dz_far(x0, x1, y0, y1, lam):
    fx, fy = max(abs(x0), abs(x1)), max(abs(y0), abs(y1))
    return 1.0 / lam - math.sqrt(max(1.0 / lam**2 - (fx * fx + fy * fy), 0.0))


@pytest.mark.parametrize("H,W,p", [(1080, 1920, 8e-6), (2160, 3840, 3.74e-6)])
def test_tile_footprint_contains_every_untruncated_pixel(H, W, p):
    rng = np.random.default_rng(21)
    TW, TH = 64, 32
    for lam in (638e-9, 450e-9):
        FX, FY, DZ = _grid(H, W, p, lam)
        dzmax = np.abs(DZ).max()
        for _ in range(40):
            q = rng.normal(size=4)
            r1, r2 = _rot(q)
            su, sv = np.exp(rng.normal(math.log(2 * p), 0.5, 2))
            M = np.array([[su * r1[0], sv * r2[0]], [su * r1[1], sv * r2[1]]])
            w = np.array([su * r1[2], sv * r2[2]])
            rho_grid = math.sqrt(TAU / (2 * math.pi**2)) + dzmax * np.linalg.norm(w)
            wz = np.linalg.norm(w) / rho_grid
            for _ in range(6):
                ty, tx = rng.integers(0, (H + TH - 1) // TH), rng.integers(0, (W + TW - 1) // TW)
                r0, c0 = ty * TH, tx * TW
                r1_, c1_ = min(r0 + TH, H), min(c0 + TW, W)
                fx, fy, dz = FX[r0:r1_, c0:c1_], FY[r0:r1_, c0:c1_], DZ[r0:r1_, c0:c1_]
                dzt = _dz_far(fx.min(), fx.max(), fy.min(), fy.max(), lam)
                assert dzt == pytest.approx(np.abs(dz).max(), rel=1e-9, abs=1e-9)  # the farthest pixel
                a = su * (r1[0] * fx + r1[1] * fy + r1[2] * dz)
                b = sv * (r2[0] * fx + r2[1] * fy + r2[2] * dz)
                E = 2 * math.pi**2 * (a * a + b * b)
                inside = E <= TAU
                mf = np.stack([M[0, 0] * fx + M[1, 0] * fy, M[0, 1] * fx + M[1, 1] * fy])
                rho_t = math.sqrt(TAU / (2 * math.pi**2)) + dzt * np.linalg.norm(w)
                # the per-tile ellipse as the kernels form it: the grid-wide one scaled by
                # 1 / (1 - (dzmax - dzt) wz)^2
                scale = 1.0 / (1.0 - (dzmax - dzt) * wz) ** 2
                q_t = (mf[0] ** 2 + mf[1] ** 2) / rho_grid**2 * scale
                assert np.all(q_t[inside] <= 1.0 + 1e-12), (lam, q_t[inside].max())
                assert (rho_t / rho_grid) ** 2 == pytest.approx(1.0 / scale, rel=1e-12)


def test_tile_bound_is_tighter_than_the_grid_bound_away_from_the_edges():
    """Tiles nearer f = 0 than the grid's corners get a smaller |d_z| bound, hence a smaller
    ellipse for tilted Gaussians (|w| > 0): the cull's saving."""
    H, W, p, lam = 1080, 1920, 8e-6, 520e-9
    FX, FY, DZ = _grid(H, W, p, lam)
    dzmax = np.abs(DZ).max()
    c = W // 2
    dzt = _dz_far(FX[0, c], FX[0, c + 63], FY[H // 2, 0], FY[H // 2 + 31, 0], lam)
    assert dzt < 0.01 * dzmax
    rho0 = math.sqrt(TAU / (2 * math.pi**2))
    wn = 20e-6  # |w| of a strongly tilted 20 um Gaussian
    assert rho0 + dzt * wn < rho0 + dzmax * wn
