"""Test-side helpers: explicit scenes and quaternion algebra (input construction only)."""
import math

import numpy as np

from paper_2505_06582_gb300.scenes import SLM, Scene


def qmul(a, b):
    """Hamilton product of quaternions (w, x, y, z)."""
    aw, ax, ay, az = a
    bw, bx, by, bz = b
    return np.array([aw * bw - ax * bx - ay * by - az * bz,
                     aw * bx + ax * bw + ay * bz - az * by,
                     aw * by - ax * bz + ay * bw + az * bx,
                     aw * bz + ax * by - ay * bx + az * bw])


def qaxis(axis, angle):
    axis = np.asarray(axis, dtype=float)
    axis = axis / np.linalg.norm(axis)
    return np.concatenate([[math.cos(angle / 2)], math.sin(angle / 2) * axis])


def rotmat(q):
    """Rotation matrix of a quaternion, built as R v = q v q* (test-side restatement)."""
    q = np.asarray(q, dtype=float) / np.linalg.norm(q)
    cols = []
    for e in np.eye(3):
        v = np.concatenate([[0.0], e])
        r = qmul(qmul(q, v), q * np.array([1, -1, -1, -1]))
        cols.append(r[1:])
    return np.stack(cols, 1)


def make_scene(means, quats, scales, opac, amps):
    means = np.asarray(means, dtype=np.float64).reshape(-1, 3)
    n = means.shape[0]
    quats = np.asarray(quats, dtype=np.float64).reshape(n, 4)
    return Scene(means, quats, np.asarray(scales, dtype=np.float64).reshape(n, 2),
                 np.asarray(opac, dtype=np.float64).reshape(n), np.asarray(amps, dtype=np.float64).reshape(n, -1))


def rel_l2(a, b):
    a = np.asarray(a)
    b = np.asarray(b)
    return float(np.linalg.norm((a - b).ravel()) / max(np.linalg.norm(b.ravel()), 1e-300))


def grid_freqs(slm: SLM, lam):
    fx = (np.arange(slm.W) - slm.W // 2) / (slm.W * slm.pitch_x)
    fy = (np.arange(slm.H) - slm.H // 2) / (slm.H * slm.pitch_y)
    FX, FY = np.meshgrid(fx, fy)
    FZ = np.sqrt(np.maximum(1.0 / lam ** 2 - FX ** 2 - FY ** 2, 0.0))
    return FX, FY, FZ
