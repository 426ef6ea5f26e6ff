"""Seeded synthetic scenes for Gaussian Wave Splatting workloads.

This module only draws inputs: Gaussian records (mean, quaternion, scales, opacity,
per-wavelength amplitude), SLM descriptions and cotangent arrays.  It contains none of
the method's arithmetic (no spectra, no propagation, no blending), so both the CUDA
path and the CPU oracle can be fed from it without sharing any computation.

Distributions follow the workloads of the paper's evaluation (2D Gaussians in a
hologram volume about 1 cm deep in front of a 1920x1080, 8 um SLM; scenes of 15k to
1M Gaussians; Sec. 5 and the supplement's hardware section), with the datasets
replaced by random surfaces because the trained scenes are not available:

* ``uniform_scene``  -- means uniform over the SLM aperture at z ~ U[z0, z1],
  quaternions uniform on S^3 (4 iid normals, normalised), log-normal scales.
* ``surface_scene``  -- means on random spheres (SLM-facing hemispheres) and tilted
  planes, each Gaussian lying in its surface's tangent plane with a random in-plane
  angle.
* ``world_scene``    -- the same kind of surfaces in the world space of a camera (the
  input of the holographics front end: a 2DGS-OIT style model with degree-3 SH opacity
  coefficients), with the view, the projective mapping and the display transform that
  maps the image to the SLM and the view depths to the hologram volume.

Units: metres.  Means are float64; everything else is float32.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

__all__ = [
    "SLM", "Scene", "uniform_scene", "surface_scene", "config_scene", "batched_sizes",
    "cotangent", "random_field", "CONFIGS", "WorldScene", "world_scene", "triangle_scene",
]


@dataclass
class SLM:
    """Hologram plane: H rows (y) by W columns (x), pixel pitch and wavelengths (m)."""
    H: int
    W: int
    pitch_x: float
    pitch_y: float
    wavelengths: tuple

    @property
    def n_lambda(self) -> int:
        return len(self.wavelengths)


@dataclass
class Scene:
    mean: np.ndarray      # float64 [N,3]
    quat: np.ndarray      # float32 [N,4]  (w, x, y, z)
    scale: np.ndarray     # float32 [N,2]  (s_u, s_v)
    opacity: np.ndarray   # float32 [N]
    amp: np.ndarray       # float32 [N, n_lambda]
    meta: dict = field(default_factory=dict)

    @property
    def n(self) -> int:
        return int(self.mean.shape[0])

    def subset(self, idx) -> "Scene":
        idx = np.asarray(idx)
        return Scene(self.mean[idx].copy(), self.quat[idx].copy(), self.scale[idx].copy(),
                     self.opacity[idx].copy(), self.amp[idx].copy(), dict(self.meta))

    def concat(self, other: "Scene") -> "Scene":
        return Scene(np.concatenate([self.mean, other.mean]), np.concatenate([self.quat, other.quat]),
                     np.concatenate([self.scale, other.scale]),
                     np.concatenate([self.opacity, other.opacity]),
                     np.concatenate([self.amp, other.amp]), dict(self.meta))


def _quat_from_frame(r1, r2, r3):
    """Unit quaternion (w,x,y,z) whose rotation matrix has columns r1, r2, r3.

    Input preparation only (builds a rotation from a drawn tangent frame)."""
    m00, m10, m20 = r1[:, 0], r1[:, 1], r1[:, 2]
    m01, m11, m21 = r2[:, 0], r2[:, 1], r2[:, 2]
    m02, m12, m22 = r3[:, 0], r3[:, 1], r3[:, 2]
    tr = m00 + m11 + m22
    q = np.zeros((r1.shape[0], 4))
    c0 = tr > 0
    s = np.sqrt(np.maximum(tr + 1.0, 1e-300)) * 2
    q[c0] = np.stack([0.25 * s, (m21 - m12) / s, (m02 - m20) / s, (m10 - m01) / s], 1)[c0]
    c1 = (~c0) & (m00 > m11) & (m00 > m22)
    s = np.sqrt(np.maximum(1.0 + m00 - m11 - m22, 1e-300)) * 2
    q[c1] = np.stack([(m21 - m12) / s, 0.25 * s, (m01 + m10) / s, (m02 + m20) / s], 1)[c1]
    c2 = (~c0) & (~c1) & (m11 > m22)
    s = np.sqrt(np.maximum(1.0 + m11 - m00 - m22, 1e-300)) * 2
    q[c2] = np.stack([(m02 - m20) / s, (m01 + m10) / s, 0.25 * s, (m12 + m21) / s], 1)[c2]
    c3 = (~c0) & (~c1) & (~c2)
    s = np.sqrt(np.maximum(1.0 + m22 - m00 - m11, 1e-300)) * 2
    q[c3] = np.stack([(m10 - m01) / s, (m02 + m20) / s, (m12 + m21) / s, 0.25 * s], 1)[c3]
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    return q


def _tangent_frame(normal, psi):
    """Right-handed frame (r1, r2, r3=normal) with in-plane angle psi."""
    n = normal / np.linalg.norm(normal, axis=1, keepdims=True)
    helper = np.where(np.abs(n[:, 2:3]) < 0.9, np.array([[0.0, 0.0, 1.0]]), np.array([[1.0, 0.0, 0.0]]))
    e1 = np.cross(helper, n)
    e1 /= np.linalg.norm(e1, axis=1, keepdims=True)
    e2 = np.cross(n, e1)
    c, s = np.cos(psi)[:, None], np.sin(psi)[:, None]
    r1 = c * e1 + s * e2
    r2 = -s * e1 + c * e2
    return r1, r2, n


def _lognormal_scales(rng, n, median, sigma_log):
    return np.exp(rng.normal(math.log(median), sigma_log, size=(n, 2))).astype(np.float32)


def uniform_scene(seed: int, n: int, slm: SLM, z_range=(1e-3, 5e-3), scale_median_px=4.0,
                  sigma_log=0.5, opacity_range=(0.2, 1.0)) -> Scene:
    """Means uniform over the aperture, quaternions uniform on S^3."""
    rng = np.random.default_rng(seed)
    ax, ay = slm.W * slm.pitch_x, slm.H * slm.pitch_y
    mean = np.empty((n, 3))
    mean[:, 0] = rng.uniform(-ax / 2, ax / 2, n)
    mean[:, 1] = rng.uniform(-ay / 2, ay / 2, n)
    mean[:, 2] = rng.uniform(z_range[0], z_range[1], n)
    q = rng.normal(size=(n, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    scale = _lognormal_scales(rng, n, scale_median_px * slm.pitch_x, sigma_log)
    opacity = rng.uniform(opacity_range[0], opacity_range[1], n).astype(np.float32)
    amp = rng.uniform(0.0, 1.0, (n, slm.n_lambda)).astype(np.float32)
    return Scene(mean, q.astype(np.float32), scale, opacity, amp, {"kind": "uniform", "seed": seed})


def surface_scene(seed: int, n: int, slm: SLM, n_surfaces=8, scale_median_px=2.0, sigma_log=0.5,
                  opacity_range=(0.05, 1.0), z_clip=(2e-3, 10e-3)) -> Scene:
    """Gaussians on random spheres (SLM-facing hemispheres) and tilted planes."""
    rng = np.random.default_rng(seed)
    if n == 0:
        z = np.zeros
        return Scene(z((0, 3)), z((0, 4), np.float32), z((0, 2), np.float32), z(0, np.float32),
                     z((0, slm.n_lambda), np.float32), {"kind": "surface", "seed": seed, "surfaces": n_surfaces})
    ax, ay = slm.W * slm.pitch_x, slm.H * slm.pitch_y
    counts = np.full(n_surfaces, n // n_surfaces)
    counts[: n - counts.sum()] += 1
    pts, nrm = [], []
    for k in range(n_surfaces):
        m = int(counts[k])
        if m == 0:
            continue
        if rng.uniform() < 0.5:  # sphere, points on the hemisphere facing the SLM (z < z_c)
            c = np.array([rng.uniform(-0.3 * ax, 0.3 * ax), rng.uniform(-0.3 * ay, 0.3 * ay),
                          rng.uniform(4e-3, 8e-3)])
            rad = rng.uniform(0.5e-3, 2e-3)
            v = rng.normal(size=(m, 3))
            v /= np.linalg.norm(v, axis=1, keepdims=True)
            v[:, 2] = -np.abs(v[:, 2])
            pts.append(c + rad * v)
            nrm.append(v)
        else:  # plane with a normal within 30 degrees of +z, a random rectangle of the aperture
            cos_t = rng.uniform(math.cos(math.radians(30.0)), 1.0)
            sin_t = math.sqrt(1.0 - cos_t * cos_t)
            phi = rng.uniform(0, 2 * math.pi)
            nv = np.array([sin_t * math.cos(phi), sin_t * math.sin(phi), cos_t])
            hx, hy = rng.uniform(0.1, 0.45) * ax, rng.uniform(0.1, 0.45) * ay
            cx, cy = rng.uniform(-ax / 2 + hx, ax / 2 - hx), rng.uniform(-ay / 2 + hy, ay / 2 - hy)
            z0 = rng.uniform(3e-3, 9e-3)
            x = rng.uniform(cx - hx, cx + hx, m)
            y = rng.uniform(cy - hy, cy + hy, m)
            z = z0 - (nv[0] * (x - cx) + nv[1] * (y - cy)) / nv[2]
            pts.append(np.stack([x, y, z], 1))
            nrm.append(np.tile(nv, (m, 1)))
    mean = np.concatenate(pts)
    normal = np.concatenate(nrm)
    mean[:, 2] = np.clip(mean[:, 2], z_clip[0], z_clip[1])
    psi = rng.uniform(0, 2 * math.pi, mean.shape[0])
    r1, r2, r3 = _tangent_frame(normal, psi)
    q = _quat_from_frame(r1, r2, r3).astype(np.float32)
    scale = _lognormal_scales(rng, mean.shape[0], scale_median_px * slm.pitch_x, sigma_log)
    opacity = rng.uniform(opacity_range[0], opacity_range[1], mean.shape[0]).astype(np.float32)
    amp = rng.uniform(0.0, 1.0, (mean.shape[0], slm.n_lambda)).astype(np.float32)
    return Scene(mean, q, scale, opacity, amp, {"kind": "surface", "seed": seed, "surfaces": n_surfaces})


@dataclass
class WorldScene:
    """World-space Gaussians of one view (front-end input) and the view / display geometry."""
    mean: np.ndarray      # float64 [N,3], world (m)
    quat: np.ndarray      # float32 [N,4] (w, x, y, z), world rotation
    scale: np.ndarray     # float32 [N,3]; surfels have scale[:, 2] = 0
    sh: np.ndarray        # float32 [N,16], degree-3 SH coefficients of the opacity
    amp: np.ndarray       # float32 [N, n_lambda]
    view: np.ndarray      # float64 [3,4]: x_view = W x_world + t, camera looking down -z
    fx: float
    fy: float
    cx: float
    cy: float
    holo: np.ndarray      # float64 [3,4]: ray space (pixels, view z) -> hologram space (m)
    meta: dict = field(default_factory=dict)

    @property
    def n(self) -> int:
        return int(self.mean.shape[0])


def _random_rotation(rng) -> np.ndarray:
    q = rng.normal(size=4)
    q /= np.linalg.norm(q)
    w, x, y, z = q
    return np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)],
                     [2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)],
                     [2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)]])


def world_scene(seed: int, n: int, slm: SLM, n_surfaces=8, depth=(1.5, 3.0), fov_deg=40.0,
                hologram_depth=(2e-3, 10e-3), scale_px=2.0, sigma_log=0.5, volume_frac=0.0,
                sh_spread=0.1) -> WorldScene:
    """Surfaces (camera-facing sphere caps and tilted planes) inside the view frustum at view
    depths ``depth`` (m), posed in the world by a random camera; surfels whose projected scales
    are about ``scale_px`` pixels.  A fraction ``volume_frac`` gets a non-zero third scale (3D
    Gaussians).  The SH opacity has a DC term for a base opacity U[0.3, 1] and higher orders
    N(0, sh_spread).  The display maps pixel (u, v) to (u - W/2) px, (v - H/2) py and the view
    depths linearly onto ``hologram_depth`` (near -> near)."""
    rng = np.random.default_rng(seed)
    W_px, H_px = slm.W, slm.H
    fx = fy = (W_px / 2) / math.tan(math.radians(fov_deg) / 2)
    cx, cy = W_px / 2, H_px / 2
    half_x, half_y = (W_px / 2) / fx, (H_px / 2) / fy  # frustum half-widths per unit depth
    counts = np.full(n_surfaces, n // n_surfaces)
    counts[: n - counts.sum()] += 1
    pts, nrm = [], []
    for k in range(n_surfaces):
        m = int(counts[k])
        if m == 0:
            continue
        d = rng.uniform(depth[0] + 0.2 * (depth[1] - depth[0]), depth[1] - 0.2 * (depth[1] - depth[0]))
        ctr = np.array([rng.uniform(-0.5, 0.5) * half_x * d, rng.uniform(-0.5, 0.5) * half_y * d, -d])
        if rng.uniform() < 0.5:  # sphere cap facing the camera (+z in view space)
            rad = rng.uniform(0.05, 0.15) * d * half_y
            v = rng.normal(size=(m, 3))
            v /= np.linalg.norm(v, axis=1, keepdims=True)
            v[:, 2] = np.abs(v[:, 2])
            pts.append(ctr + rad * v)
            nrm.append(v)
        else:  # plane patch, normal within 45 degrees of the view axis
            cos_t = rng.uniform(math.cos(math.radians(45.0)), 1.0)
            sin_t = math.sqrt(1.0 - cos_t * cos_t)
            phi = rng.uniform(0, 2 * math.pi)
            nv = np.array([sin_t * math.cos(phi), sin_t * math.sin(phi), cos_t])
            hx, hy = rng.uniform(0.1, 0.3) * half_x * d, rng.uniform(0.1, 0.3) * half_y * d
            x = rng.uniform(ctr[0] - hx, ctr[0] + hx, m)
            y = rng.uniform(ctr[1] - hy, ctr[1] + hy, m)
            z = ctr[2] - (nv[0] * (x - ctr[0]) + nv[1] * (y - ctr[1])) / nv[2]
            pts.append(np.stack([x, y, z], 1))
            nrm.append(np.tile(nv, (m, 1)))
    if n > 0:
        xv = np.concatenate(pts)
        normal = np.concatenate(nrm)
    else:
        xv, normal = np.zeros((0, 3)), np.zeros((0, 3))
    xv[:, 2] = np.clip(xv[:, 2], -depth[1], -depth[0])
    psi = rng.uniform(0, 2 * math.pi, xv.shape[0])
    r1, r2, r3 = _tangent_frame(normal, psi) if n > 0 else (normal, normal, normal)
    # camera pose: x_view = Rc x_world + t  <=>  x_world = Rc^T (x_view - t)
    Rc = _random_rotation(rng)
    t = rng.normal(size=3)
    view = np.concatenate([Rc, t[:, None]], axis=1)
    mean = (xv - t) @ Rc
    frame = np.stack([r1, r2, r3], axis=2)  # view-space columns
    wframe = np.einsum("ji,njk->nik", Rc, frame)  # Rc^T [r1 r2 r3]
    q = _quat_from_frame(wframe[:, :, 0], wframe[:, :, 1], wframe[:, :, 2]).astype(np.float32) if n > 0 \
        else np.zeros((0, 4), np.float32)
    px_world = (-xv[:, 2]) / fx  # metres per pixel at each depth
    s2 = np.exp(rng.normal(math.log(scale_px), sigma_log, (xv.shape[0], 2))) * px_world[:, None]
    s3 = np.where(rng.uniform(size=xv.shape[0]) < volume_frac, 0.5 * s2.min(axis=1), 0.0)
    scale = np.concatenate([s2, s3[:, None]], axis=1).astype(np.float32)
    sh = rng.normal(0.0, sh_spread, (xv.shape[0], 16))
    sh[:, 0] = rng.uniform(0.3, 1.0, xv.shape[0]) * 2.0 * math.sqrt(math.pi)  # Y_00 = 1 / (2 sqrt(pi))
    amp = rng.uniform(0.0, 1.0, (xv.shape[0], slm.n_lambda)).astype(np.float32)
    a = (hologram_depth[1] - hologram_depth[0]) / (depth[0] - depth[1])  # view z = -depth
    bz = hologram_depth[0] + a * depth[0]
    holo = np.array([[slm.pitch_x, 0.0, 0.0, -cx * slm.pitch_x],
                     [0.0, slm.pitch_y, 0.0, -cy * slm.pitch_y],
                     [0.0, 0.0, a, bz]])
    return WorldScene(mean, q, scale, sh.astype(np.float32), amp, view, fx, fy, cx, cy, holo,
                      {"kind": "world", "seed": seed, "surfaces": n_surfaces})


def triangle_scene(seed: int, n: int, slm: SLM, size_px=3.0, **surface_kw):
    """Triangle soup (vertices float64 [n,3,3], opacity float32 [n], amp float32 [n, n_lambda]):
    one small triangle per point of ``surface_scene`` in its tangent plane, random shape, edges
    about ``size_px`` pixels."""
    sc = surface_scene(seed, n, slm, **surface_kw)
    rng = np.random.default_rng(seed + 7919)
    q = sc.quat.astype(np.float64)
    w, x, y, z = q[:, 0], q[:, 1], q[:, 2], q[:, 3]
    r1 = np.stack([1 - 2 * (y * y + z * z), 2 * (x * y + w * z), 2 * (x * z - w * y)], 1)
    r2 = np.stack([2 * (x * y - w * z), 1 - 2 * (x * x + z * z), 2 * (y * z + w * x)], 1)
    ang = rng.uniform(0, 2 * math.pi, (sc.n, 3)) + np.array([0.0, 2.1, 4.2])
    rad = size_px * slm.pitch_x * rng.uniform(0.5, 1.2, (sc.n, 3))
    verts = sc.mean[:, None, :] + rad[:, :, None] * (np.cos(ang)[:, :, None] * r1[:, None, :]
                                                     + np.sin(ang)[:, :, None] * r2[:, None, :])
    return verts, sc.opacity, sc.amp


RGB = (638e-9, 520e-9, 450e-9)

# name -> (slm, generator kwargs).  Sizes and distributions of the five workloads.
CONFIGS = {
    "c0_plain_fp64": dict(slm=SLM(128, 128, 8e-6, 8e-6, (520e-9,)), kind="uniform", seed=0, n=64),
    "c1_slm_size": dict(slm=SLM(1080, 1920, 8e-6, 8e-6, RGB), kind="surface", seed=1, n=20_000, n_surfaces=8),
    "c2_precision_at_scale": dict(slm=SLM(2160, 3840, 3.74e-6, 3.74e-6, RGB), kind="surface", seed=2,
                                  n=1_000_000, n_surfaces=32),
    "c4_differentiable": dict(slm=SLM(1080, 1920, 8e-6, 8e-6, RGB), kind="surface", seed=4, n=100_000,
                              n_surfaces=8),
    "headline_1m_1080p_3l": dict(slm=SLM(1080, 1920, 8e-6, 8e-6, RGB), kind="surface", seed=1,
                                 n=1_000_000, n_surfaces=32),
    "paper_tab3_1024x1280": dict(slm=SLM(1024, 1280, 8e-6, 8e-6, (520e-9,)), kind="surface", seed=5,
                                 n=15_000, n_surfaces=8),
    "paper_tab3_2000x2000": dict(slm=SLM(2000, 2000, 8e-6, 8e-6, (520e-9,)), kind="surface", seed=5,
                                 n=15_000, n_surfaces=8),
}


def config_scene(name: str, n: int | None = None, seed: int | None = None):
    """(scene, slm) for a named workload; ``n`` overrides the Gaussian count."""
    cfg = CONFIGS[name]
    slm = cfg["slm"]
    n = cfg["n"] if n is None else n
    seed = cfg["seed"] if seed is None else seed
    if cfg["kind"] == "uniform":
        return uniform_scene(seed, n, slm), slm
    return surface_scene(seed, n, slm, n_surfaces=cfg.get("n_surfaces", 8)), slm


def batched_sizes(n_scenes=64, lo=1_000, hi=200_000, seed=3):
    """Scene sizes log-uniform in [lo, hi] (the batched multi-scene workload)."""
    rng = np.random.default_rng(seed)
    return [int(round(math.exp(rng.uniform(math.log(lo), math.log(hi))))) for _ in range(n_scenes)]


def batched_scenes(slm: SLM, n_scenes=64, lo=1_000, hi=200_000, seed=3):
    sizes = batched_sizes(n_scenes, lo, hi, seed)
    return [surface_scene(seed + k, sizes[k], slm) for k in range(n_scenes)]


def cotangent(seed: int, slm: SLM, dtype=np.complex64) -> np.ndarray:
    """Seeded complex normal array [n_lambda][H][W] (a synthetic upstream gradient)."""
    rng = np.random.default_rng(seed)
    shape = (slm.n_lambda, slm.H, slm.W)
    return (rng.standard_normal(shape) + 1j * rng.standard_normal(shape)).astype(dtype)


def random_field(seed: int, shape, dtype=np.complex128, zero_frac=0.0) -> np.ndarray:
    """Seeded complex field with log-normal amplitudes and uniform phases."""
    rng = np.random.default_rng(seed)
    a = np.exp(rng.normal(0.0, 1.0, shape))
    ph = rng.uniform(-math.pi, math.pi, shape)
    f = a * np.exp(1j * ph)
    if zero_frac > 0:
        f[rng.uniform(size=shape) < zero_frac] = 0
    return f.astype(dtype)
