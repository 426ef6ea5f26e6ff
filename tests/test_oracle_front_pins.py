"""Pins of the holographics front-end oracle (Supplement Sec. 1.1) and of the SH opacity (Sec. 4.2).

Each pin checks the oracle against something other than itself: quadrature orthonormality and
the addition theorem of the spherical harmonics, finite differences of the projective mapping,
Monte-Carlo moments of Gaussians pushed through the transforms, special cases that reduce to
the identity, and the factorisation Sigma = R S S^T R^T.
"""
import numpy as np
import pytest

from oracle import holographics as H


def _dirs(rng, n):
    d = rng.normal(size=(n, 3))
    return d / np.linalg.norm(d, axis=1, keepdims=True)


def _view(rng):
    q = rng.normal(size=4)
    W = H.rotation(q[None])[0]
    t = rng.normal(size=3) * 0.1
    return np.concatenate([W, t[:, None]], axis=1)


# ---- spherical harmonics ------------------------------------------------------------------

def test_sh_orthonormal_quadrature():
    # Gauss-Legendre in cos(theta) x uniform phi: exact for the degree-6 products of two
    # degree-3 harmonics, so any wrong constant or polynomial shows up
    xg, wg = np.polynomial.legendre.leggauss(16)
    nphi = 32
    phi = (np.arange(nphi) + 0.5) * 2 * np.pi / nphi
    ct, ph = np.meshgrid(xg, phi, indexing="ij")
    st = np.sqrt(1 - ct ** 2)
    d = np.stack([st * np.cos(ph), st * np.sin(ph), ct], axis=-1).reshape(-1, 3)
    w = (wg[:, None] * np.full(nphi, 2 * np.pi / nphi)[None, :]).reshape(-1)
    Y = H.sh_basis(d, 3)
    G = (Y * w[:, None]).T @ Y
    assert np.abs(G - np.eye(16)).max() < 1e-13


def test_sh_addition_theorem():
    # sum_m Y_lm(d) Y_lm(d') = (2l + 1) / (4 pi) P_l(d . d')
    rng = np.random.default_rng(1)
    d, e = _dirs(rng, 50), _dirs(rng, 50)
    Yd, Ye = H.sh_basis(d, 3), H.sh_basis(e, 3)
    c = np.sum(d * e, axis=1)
    for l in range(4):
        sl = slice(l * l, (l + 1) ** 2)
        lhs = np.sum(Yd[:, sl] * Ye[:, sl], axis=1)
        Pl = np.polynomial.legendre.legval(c, [0] * l + [1])
        assert np.abs(lhs - (2 * l + 1) / (4 * np.pi) * Pl).max() < 1e-13


def test_sh_sign_convention():
    # Condon-Shortley phase, m = -l..l: Y_1 = sqrt(3/4pi) (-y, z, -x); Y_2,-2 = +sqrt(15/4pi) xy
    c1 = np.sqrt(3 / (4 * np.pi))
    Y = H.sh_basis(np.eye(3), 3)
    # rows: d = e_x, e_y, e_z; columns: m = -1, 0, 1
    assert np.allclose(Y[:, 1:4], c1 * np.array([[0, 0, -1], [-1, 0, 0], [0, 1, 0]]))
    xy = np.array([[np.sqrt(0.5), np.sqrt(0.5), 0.0]])
    assert np.isclose(H.sh_basis(xy, 2)[0, 4], np.sqrt(15 / (4 * np.pi)) * 0.5)


def test_camera_centre_maps_to_the_view_origin():
    rng = np.random.default_rng(12)
    for _ in range(5):
        view = _view(rng)
        assert np.allclose(view[:, :3] @ H.camera_centre(view) + view[:, 3], 0.0, atol=1e-14)


def test_view_opacity_direction_and_clamp():
    # the degree-0 term is view-independent; a pure l = 1, m = 0 term follows d_z of the viewing
    # direction from the camera centre, and the result is clamped to [0, 1]
    rng = np.random.default_rng(2)
    view = _view(rng)
    c = np.linalg.solve(view[:, :3], -view[:, 3])  # the point the view maps to its origin
    mean = c[None, :] + _dirs(rng, 64) * rng.uniform(0.5, 2.0, (64, 1))
    sh = np.zeros((64, 16))
    sh[:, 0] = 0.5 * 2 * np.sqrt(np.pi)
    assert np.allclose(H.view_opacity(sh, mean, view, 0), 0.5)
    sh[:, 2] = 0.3 / np.sqrt(3 / (4 * np.pi))
    d = (mean - c) / np.linalg.norm(mean - c, axis=1, keepdims=True)
    assert np.allclose(H.view_opacity(sh, mean, view, 1), np.clip(0.5 + 0.3 * d[:, 2], 0, 1), atol=1e-14)
    sh[:, 0] = 5.0
    assert np.all(H.view_opacity(sh, mean, view, 3) == 1.0)


# ---- geometric pipeline -----------------------------------------------------------------

@pytest.mark.parametrize("proj", [H.PROJ_PERSPECTIVE, H.PROJ_ORTHOGRAPHIC])
def test_jacobian_is_the_derivative_of_phi(proj):
    rng = np.random.default_rng(3)
    xv = rng.normal(size=(20, 3))
    xv[:, 2] = -rng.uniform(0.5, 3.0, 20)
    fx, fy, cx, cy = 800.0, 700.0, 320.0, 240.0
    _, J = H.project(xv, fx, fy, cx, cy, proj)
    h = 1e-6
    for k in range(3):
        e = np.zeros(3)
        e[k] = h
        up, _ = H.project(xv + e, fx, fy, cx, cy, proj)
        um, _ = H.project(xv - e, fx, fy, cx, cy, proj)
        fd = (up - um) / (2 * h)
        assert np.allclose(J[:, :, k], fd, rtol=1e-6, atol=1e-6 * max(fx, fy))


def test_identity_pipeline_keeps_an_untilted_surfel():
    # identity view, orthographic unit mapping, identity hologram transform: a surfel
    # parallel to the xy plane comes out unchanged (mean, in-plane covariance, scales)
    rng = np.random.default_rng(4)
    n = 30
    ang = rng.uniform(-np.pi, np.pi, n)
    q = np.stack([np.cos(ang / 2), 0 * ang, 0 * ang, np.sin(ang / 2)], axis=1)  # about z
    s = np.stack([rng.uniform(1, 3, n), rng.uniform(0.2, 1, n), np.zeros(n)], axis=1)
    mean = rng.normal(size=(n, 3))
    mean[:, 2] = -rng.uniform(1, 2, n)
    view = np.concatenate([np.eye(3), np.zeros((3, 1))], axis=1)
    holo = np.concatenate([np.eye(3), np.zeros((3, 1))], axis=1)
    out = H.holographics(mean, q, s, view, 1.0, 1.0, 0.0, 0.0, H.PROJ_ORTHOGRAPHIC, 0.0, holo)
    assert out["valid"].all()
    assert np.allclose(out["mean"], mean, atol=1e-14)
    assert np.allclose(out["scale"], s[:, :2], rtol=1e-12)
    R = H.rotation(q)
    sig = np.einsum("nik,nk,njk->nij", R, s ** 2, R)
    assert np.allclose(out["sigma"], sig, atol=1e-12)


def test_orthographic_chain_matches_monte_carlo_moments():
    # orthographic projection and affine hologram transform are linear, so the lifted covariance
    # must be the covariance of world samples pushed through view, projection, depth collapse
    # and A (an independent check of every matrix product and transpose in the chain)
    rng = np.random.default_rng(5)
    view = _view(rng)
    holo = np.concatenate([rng.normal(size=(3, 3)), rng.normal(size=(3, 1))], axis=1)
    q = rng.normal(size=(1, 4))
    s = np.array([[0.3, 0.1, 0.05]])
    mean = (H.camera_centre(view) - 3 * view[2, :3])[None, :]  # on the optical axis, 3 in front
    fx, fy, cx, cy = 2.0, 1.5, 0.1, -0.2
    out = H.holographics(mean, q, s, view, fx, fy, cx, cy, H.PROJ_ORTHOGRAPHIC, 0.0, holo)
    m = 400_000
    R = H.rotation(q)[0]
    xw = mean + (rng.normal(size=(m, 3)) * s) @ R.T
    xv = xw @ view[:, :3].T + view[:, 3]
    uv = np.stack([fx * xv[:, 0] + cx, fy * xv[:, 1] + cy], axis=1)
    zv = np.full((m, 1), (mean @ view[:, :3].T + view[:, 3])[0, 2])  # lifted: the mean's depth
    y = np.concatenate([uv, zv], axis=1) @ holo[:, :3].T + holo[:, 3]
    cov = np.cov(y.T)
    scale = np.abs(out["sigma"][0]).max()
    assert np.abs(cov - out["sigma"][0]).max() < 0.02 * scale
    assert np.allclose(y.mean(axis=0), out["mean"][0], atol=0.01 * np.sqrt(scale))


def test_perspective_ewa_matches_projected_samples_of_a_small_gaussian():
    # for a Gaussian small against its depth the local affine (EWA) approximation is tight:
    # the covariance of the truly projected samples matches J W Sigma_w W^T J^T
    rng = np.random.default_rng(6)
    view = _view(rng)
    c = H.camera_centre(view)
    mean = (c + 5.0 * (-view[2, :3]) + 0.8 * view[0, :3])[None, :]
    q = rng.normal(size=(1, 4))
    s = np.array([[0.02, 0.01, 0.005]])
    holo = np.concatenate([np.eye(3), np.zeros((3, 1))], axis=1)
    fx, fy, cx, cy = 1000.0, 900.0, 0.0, 0.0
    out = H.holographics(mean, q, s, view, fx, fy, cx, cy, H.PROJ_PERSPECTIVE, 0.1, holo)
    m = 400_000
    R = H.rotation(q)[0]
    xw = mean + (rng.normal(size=(m, 3)) * s) @ R.T
    xv = xw @ view[:, :3].T + view[:, 3]
    uv, _ = H.project(xv, fx, fy, cx, cy, H.PROJ_PERSPECTIVE)
    cov = np.cov(uv.T)
    ref = out["sigma2d"][0]
    assert np.abs(cov - ref).max() < 0.02 * np.abs(ref).max()


def test_factorisation_reproduces_the_lifted_covariance():
    # Sigma = A [[Sigma_2D, 0], [0, 0]] A^T must equal R diag(s_u^2, s_v^2, 0) R^T with R a
    # proper rotation (from the quaternion) and s_u >= s_v
    rng = np.random.default_rng(7)
    n = 200
    view = _view(rng)
    c = H.camera_centre(view)
    mean = c + (-view[2, :3])[None, :] * rng.uniform(1, 4, (n, 1)) + rng.normal(size=(n, 3)) * 0.3
    q = rng.normal(size=(n, 4))
    s = np.abs(rng.normal(size=(n, 3))) * 0.05
    s[: n // 2, 2] = 0.0  # 2D surfels
    holo = np.concatenate([np.diag([1e-5, 1e-5, 2e-3]) + 1e-7 * rng.normal(size=(3, 3)),
                           rng.normal(size=(3, 1)) * 1e-3], axis=1)
    out = H.holographics(mean, q, s, view, 900.0, 900.0, 0.0, 0.0, H.PROJ_PERSPECTIVE, 0.1, holo)
    A = holo[:, :3]
    lifted = np.zeros((n, 3, 3))
    lifted[:, :2, :2] = out["sigma2d"]
    direct = A[None] @ lifted @ A.T[None]
    R = H.rotation(out["quat"])
    sc = out["scale"]
    rebuilt = np.einsum("nik,nk,njk->nij", R[:, :, :2], sc ** 2, R[:, :, :2])
    tol = 1e-10 * np.abs(direct).max(axis=(1, 2))
    assert np.all(np.abs(rebuilt - direct).max(axis=(1, 2)) <= tol)
    assert np.all(sc[:, 0] >= sc[:, 1])
    assert np.allclose(np.linalg.det(R), 1.0)
    assert np.all(out["quat"][:, 0] >= 0)


def test_mean_chain_and_culling():
    # mu = A (phi(W mu_w + t), (W mu_w + t)_z) + b; behind the camera (or closer than z_near)
    # the Gaussian is culled
    view = np.concatenate([np.eye(3), np.array([[0.0], [0.0], [-2.0]])], axis=1)  # camera at z = 2
    holo = np.concatenate([np.diag([2.0, 3.0, -1.0]), np.array([[1.0], [2.0], [0.5]])], axis=1)
    mean = np.array([[0.5, -0.25, 0.0], [0.0, 0.0, 1.95], [0.0, 0.0, 3.0]])
    q = np.tile([1.0, 0, 0, 0], (3, 1))
    s = np.tile([0.1, 0.1, 0.0], (3, 1))
    out = H.holographics(mean, q, s, view, 100.0, 100.0, 5.0, 6.0, H.PROJ_PERSPECTIVE, 0.1, holo)
    # first Gaussian: x_v = (0.5, -0.25, -2): phi = (100 * 0.5 / 2 + 5, 100 * -0.25 / 2 + 6) = (30, -6.5)
    assert np.allclose(out["mean"][0], [2 * 30 + 1, 3 * -6.5 + 2, -1 * -2.0 + 0.5])
    assert out["valid"].tolist() == [True, False, False]
