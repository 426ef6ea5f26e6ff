"""FP64 oracle of the holographics front end and of the view-dependent opacity.

TEST INFRASTRUCTURE ONLY (tests, smoke check, CPU baseline of the benchmark): the product
path never imports this module.

Follows, step by step and in the paper's order (plain numpy, float64, vectorised over N):

* Supplement Sec. 1.1 "Geometric pipeline":
  - model transform: canonical -> world, Sigma_w = R_w S_w S_w^T R_w^T (3 scales; a 2D
    surfel has a zero third scale);
  - view transform x_v = W x_w + t (camera looking down -z) and the projective mapping
    phi to ray space with the local affine (EWA) Jacobian J of phi at the mean:
    Sigma_2D = J W Sigma_w W^T J^T;
  - lifting: eigendecomposition Sigma_2D = R' S'^2 R'^T, R_v = diag(R', 1), S_v = [S'; 0]
    (zero rotation about x and y, zero z-scale), mu_v = (phi(W mu_w + t), (W mu_w + t)_z);
  - hologram transform, affine [A | b]: Sigma = A Sigma_v A^T, mu = A mu_v + b;
  - unified transformation Sigma = T T^T = R S S^T R^T (factored here by a symmetric
    eigendecomposition of the 3x3 Sigma).
* Sec. 4.2 (view-dependent opacity): alpha_i = G_i * SH(o_i, d), SH the linear real
  spherical-harmonics operator of degree <= 3 (16 coefficients), d the unit viewing
  direction from the camera centre to the Gaussian's mean in world space.

Readings where the paper is silent (listed in the design notes): perspective mapping
phi(x, y, z) = (fx x / (-z) + cx, fy y / (-z) + cy), orthographic (fx x + cx, fy y + cy);
Gaussians with view depth -z below z_near are culled (valid = False); the real SH basis and
its sign convention are those of the common 3D Gaussian splatting codes (Condon-Shortley
phase, m = -l..l); the SH opacity is clamped to [0, 1]; the scales come out descending
(s_u >= s_v), r3 = r1 x r2, and the quaternion has w >= 0.
"""
from __future__ import annotations

import numpy as np

PROJ_PERSPECTIVE, PROJ_ORTHOGRAPHIC = 0, 1


# ---- rotations --------------------------------------------------------------------------

def rotation(q):
    """Rotation matrices [n, 3, 3] (columns r1, r2, r3) of quaternions (w, x, y, z), normalised."""
    q = np.asarray(q, dtype=np.float64)
    q = q / np.linalg.norm(q, axis=-1, keepdims=True)
    w, x, y, z = q[..., 0], q[..., 1], q[..., 2], q[..., 3]
    R = np.empty(q.shape[:-1] + (3, 3))
    R[..., 0, 0] = 1 - 2 * (y * y + z * z)
    R[..., 1, 0] = 2 * (x * y + w * z)
    R[..., 2, 0] = 2 * (x * z - w * y)
    R[..., 0, 1] = 2 * (x * y - w * z)
    R[..., 1, 1] = 1 - 2 * (x * x + z * z)
    R[..., 2, 1] = 2 * (y * z + w * x)
    R[..., 0, 2] = 2 * (x * z + w * y)
    R[..., 1, 2] = 2 * (y * z - w * x)
    R[..., 2, 2] = 1 - 2 * (x * x + y * y)
    return R


def quaternion(R):
    """Unit quaternion (w, x, y, z), w >= 0, of rotation matrices [n, 3, 3]: the eigenvector of
    eigenvalue 3 of the symmetric 4x4 matrix K(R) (Bar-Itzhack's form), by numpy's eigh."""
    R = np.asarray(R, dtype=np.float64)
    n = R.shape[0]
    K = np.empty((n, 4, 4))
    Rxx, Rxy, Rxz = R[:, 0, 0], R[:, 0, 1], R[:, 0, 2]
    Ryx, Ryy, Ryz = R[:, 1, 0], R[:, 1, 1], R[:, 1, 2]
    Rzx, Rzy, Rzz = R[:, 2, 0], R[:, 2, 1], R[:, 2, 2]
    # K = (1/3) [[Rxx-Ryy-Rzz, Ryx+Rxy, Rzx+Rxz, Ryz-Rzy], ...] in (x, y, z, w) order
    K[:, 0, 0] = Rxx - Ryy - Rzz
    K[:, 0, 1] = K[:, 1, 0] = Ryx + Rxy
    K[:, 0, 2] = K[:, 2, 0] = Rzx + Rxz
    K[:, 0, 3] = K[:, 3, 0] = Rzy - Ryz
    K[:, 1, 1] = Ryy - Rxx - Rzz
    K[:, 1, 2] = K[:, 2, 1] = Rzy + Ryz
    K[:, 1, 3] = K[:, 3, 1] = Rxz - Rzx
    K[:, 2, 2] = Rzz - Rxx - Ryy
    K[:, 2, 3] = K[:, 3, 2] = Ryx - Rxy
    K[:, 3, 3] = Rxx + Ryy + Rzz
    K /= 3.0
    _, V = np.linalg.eigh(K)
    v = V[:, :, -1]  # largest eigenvalue (= 1 for a rotation)
    q = np.stack([v[:, 3], v[:, 0], v[:, 1], v[:, 2]], axis=1)
    q *= np.where(q[:, :1] < 0, -1.0, 1.0)
    return q


# ---- spherical harmonics (Sec. 4.2) ------------------------------------------------------

def sh_basis(d, degree):
    """Real spherical harmonics Y_k(d), k = l^2 + l + m, for unit directions d [n, 3], degree 0..3.

    Normalised (integral of Y_k^2 over the sphere = 1), Condon-Shortley phase, m = -l..l:
      l = 0: 1 / (2 sqrt(pi))
      l = 1: sqrt(3/4pi) (-y, z, -x)
      l = 2: sqrt(15/4pi) xy, -sqrt(15/4pi) yz, sqrt(5/16pi) (3z^2 - 1), -sqrt(15/4pi) xz, sqrt(15/16pi) (x^2 - y^2)
      l = 3: -sqrt(35/32pi) y (3x^2 - y^2), sqrt(105/4pi) xyz, -sqrt(21/32pi) y (5z^2 - 1),
             sqrt(7/16pi) z (5z^2 - 3), -sqrt(21/32pi) x (5z^2 - 1), sqrt(105/16pi) z (x^2 - y^2),
             -sqrt(35/32pi) x (x^2 - 3y^2)
    """
    d = np.asarray(d, dtype=np.float64)
    x, y, z = d[:, 0], d[:, 1], d[:, 2]
    pi = np.pi
    out = [np.full_like(x, 0.5 / np.sqrt(pi))]
    if degree >= 1:
        c1 = np.sqrt(3 / (4 * pi))
        out += [-c1 * y, c1 * z, -c1 * x]
    if degree >= 2:
        a, b, c = np.sqrt(15 / (4 * pi)), np.sqrt(5 / (16 * pi)), np.sqrt(15 / (16 * pi))
        out += [a * x * y, -a * y * z, b * (3 * z * z - 1), -a * x * z, c * (x * x - y * y)]
    if degree >= 3:
        a, b = np.sqrt(35 / (32 * pi)), np.sqrt(105 / (4 * pi))
        c, e, f = np.sqrt(21 / (32 * pi)), np.sqrt(7 / (16 * pi)), np.sqrt(105 / (16 * pi))
        out += [-a * y * (3 * x * x - y * y), b * x * y * z, -c * y * (5 * z * z - 1), e * z * (5 * z * z - 3),
                -c * x * (5 * z * z - 1), f * z * (x * x - y * y), -a * x * (x * x - 3 * y * y)]
    return np.stack(out, axis=1)


def camera_centre(view):
    """World position of the camera of the 3x4 view matrix [W | t]: c = -W^T t."""
    V = np.asarray(view, dtype=np.float64).reshape(3, 4)
    return -V[:, :3].T @ V[:, 3]


def view_opacity(sh, mean_w, view, degree):
    """alpha's opacity factor SH(o_i, d_i) (Sec. 4.2), clamped to [0, 1]; d_i = unit(mu_w - c)."""
    sh = np.asarray(sh, dtype=np.float64)
    d = np.asarray(mean_w, dtype=np.float64) - camera_centre(view)[None, :]
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    K = (degree + 1) ** 2
    o = np.sum(sh[:, :K] * sh_basis(d, degree), axis=1)
    return np.clip(o, 0.0, 1.0)


# ---- geometric pipeline (Supplement Sec. 1.1) ---------------------------------------------

def project(xv, fx, fy, cx, cy, projection):
    """Projective mapping phi of view-space points xv [n, 3] and its Jacobian J [n, 2, 3]."""
    x, y, z = xv[:, 0], xv[:, 1], xv[:, 2]
    n = xv.shape[0]
    J = np.zeros((n, 2, 3))
    if projection == PROJ_PERSPECTIVE:
        u = fx * x / (-z) + cx
        v = fy * y / (-z) + cy
        J[:, 0, 0] = fx / (-z)
        J[:, 0, 2] = fx * x / (z * z)
        J[:, 1, 1] = fy / (-z)
        J[:, 1, 2] = fy * y / (z * z)
    elif projection == PROJ_ORTHOGRAPHIC:
        u = fx * x + cx
        v = fy * y + cy
        J[:, 0, 0] = fx
        J[:, 1, 1] = fy
    else:
        raise ValueError("projection")
    return np.stack([u, v], axis=1), J


def holographics(mean_w, quat_w, scale_w, view, fx, fy, cx, cy, projection, z_near, holo):
    """World-space Gaussians -> hologram-space (mu, q, s_u, s_v) inputs of the splat.

    mean_w [n,3], quat_w [n,4] (w, x, y, z), scale_w [n,3]; view = 3x4 [W | t]; holo = 3x4 [A | b].
    Returns a dict: mean [n,3], quat [n,4], scale [n,2], sigma [n,3,3] (hologram-space
    covariance), sigma2d [n,2,2], valid [n] (False: culled, view depth below z_near).
    """
    mean_w = np.asarray(mean_w, dtype=np.float64)
    n = mean_w.shape[0]
    V = np.asarray(view, dtype=np.float64).reshape(3, 4)
    Wm, t = V[:, :3], V[:, 3]
    T = np.asarray(holo, dtype=np.float64).reshape(3, 4)
    A, b = T[:, :3], T[:, 3]
    # model transform: Sigma_w = R_w S_w S_w^T R_w^T
    Rw = rotation(quat_w)
    Sw = np.zeros((n, 3, 3))
    s = np.asarray(scale_w, dtype=np.float64)
    for k in range(3):
        Sw[:, k, k] = s[:, k]
    RS = Rw @ Sw
    sigma_w = RS @ np.transpose(RS, (0, 2, 1))
    # view transform and projective mapping (local affine approximation at the mean)
    xv = mean_w @ Wm.T + t
    valid = -xv[:, 2] >= z_near
    safe = xv.copy()
    safe[~valid, 2] = -1.0  # keep the arithmetic finite for culled Gaussians
    uv, J = project(safe, fx, fy, cx, cy, projection)
    JW = J @ Wm
    sigma2 = JW @ sigma_w @ np.transpose(JW, (0, 2, 1))
    sigma2 = 0.5 * (sigma2 + np.transpose(sigma2, (0, 2, 1)))
    # lifting: Sigma_2D = R' S'^2 R'^T, R_v = diag(R', 1), S_v = [S'; 0]
    lam, Rp = np.linalg.eigh(sigma2)           # ascending
    lam, Rp = lam[:, ::-1], Rp[:, :, ::-1]      # descending: s'_1 >= s'_2
    flip = np.linalg.det(Rp) < 0
    Rp[flip, :, 1] *= -1.0
    Sp = np.sqrt(np.maximum(lam, 0.0))
    Rv = np.zeros((n, 3, 3))
    Rv[:, :2, :2] = Rp
    Rv[:, 2, 2] = 1.0
    Sv = np.zeros((n, 3, 2))
    Sv[:, 0, 0] = Sp[:, 0]
    Sv[:, 1, 1] = Sp[:, 1]
    mu_v = np.concatenate([uv, xv[:, 2:3]], axis=1)
    # hologram transform and the unified factor T = A R_v S_v (Sigma = T T^T)
    Tf = A[None, :, :] @ Rv @ Sv
    sigma = Tf @ np.transpose(Tf, (0, 2, 1))
    mean = mu_v @ A.T + b
    # Sigma = R S S^T R^T: the two non-zero eigenpairs of Sigma; r3 = r1 x r2
    ev, U = np.linalg.eigh(sigma)                # ascending: [~0, s_v^2, s_u^2]
    r1, r2 = U[:, :, 2], U[:, :, 1]
    r3 = np.cross(r1, r2)
    R = np.stack([r1, r2, r3], axis=2)
    scale = np.sqrt(np.maximum(ev[:, [2, 1]], 0.0))
    quat = quaternion(R)
    return {"mean": mean, "quat": quat, "scale": scale, "sigma": sigma, "sigma2d": sigma2, "valid": valid}
