"""CPU checks of the differentiable workload's loss (paper_2505_06582_gb300.refocus): the refocused
intensity against a direct evaluation of the centred DFT / angular-spectrum transfer / centred
inverse DFT on a tiny grid, and the field cotangent against central differences."""
import math

import numpy as np
import torch

from paper_2505_06582_gb300 import refocus
from paper_2505_06582_gb300.scenes import SLM, random_field


def _direct_intensity(u, slm, zs):
    """|sum_f [sum_x u(x) e^{-j2pi f.x}] e^{j2pi z f_z} e^{+j2pi f.x'}|^2 by explicit sums (unscaled)."""
    H, W = slm.H, slm.W
    xs = (np.arange(W) - W // 2) * slm.pitch_x
    ys = (np.arange(H) - H // 2) * slm.pitch_y
    fx = (np.arange(W) - W // 2) / (W * slm.pitch_x)
    fy = (np.arange(H) - H // 2) / (H * slm.pitch_y)
    Ex = np.exp(-2j * math.pi * np.outer(fx, xs))  # [f][x]
    Ey = np.exp(-2j * math.pi * np.outer(fy, ys))
    out = np.zeros((slm.n_lambda, len(zs), H, W))
    for l, lam in enumerate(slm.wavelengths):
        U = Ey @ u[l] @ Ex.T
        FX, FY = np.meshgrid(fx, fy)
        k2 = 1 / lam ** 2 - FX ** 2 - FY ** 2
        for k, z in enumerate(zs):
            Uz = U * np.where(k2 > 0, np.exp(2j * math.pi * z * np.sqrt(np.maximum(k2, 0))), 0)
            uz = Ey.conj().T @ Uz @ Ex.conj() / (H * W)
            out[l, k] = np.abs(uz) ** 2
    return out


def test_refocused_intensity_matches_direct_sums():
    slm = SLM(6, 8, 8e-6, 6e-6, (638e-9, 450e-9))
    zs = (2e-3, 5e-3)
    u = random_field(1, (2, 6, 8))
    Hz = refocus.transfer(slm, zs, "cpu", dtype=torch.complex128)
    got = refocus.refocused_intensity(torch.as_tensor(u), Hz).numpy()
    want = _direct_intensity(u, slm, zs)
    assert np.abs(got - want).max() < 1e-12 * np.abs(want).max()


def test_field_cotangent_matches_central_differences():
    slm = SLM(6, 8, 8e-6, 8e-6, (520e-9,))
    zs = (2e-3, 5e-3, 8e-3)
    u = torch.as_tensor(random_field(2, (1, 6, 8)))
    Hz = refocus.transfer(slm, zs, "cpu", dtype=torch.complex128)
    t = refocus.seeded_targets(4, u, Hz).to(torch.float64)
    L, g = refocus.field_cotangent(u, Hz, t)
    v = torch.as_tensor(random_field(3, (1, 6, 8)))
    h = 1e-6
    fd = (refocus.loss(u + h * v, Hz, t) - refocus.loss(u - h * v, Hz, t)) / (2 * h)
    # PyTorch's convention: grad = dL/dRe + j dL/dIm, so dL(u + h v)/dh = Re(sum conj(grad) v)
    assert abs(float(fd) - float((g.conj() * v).real.sum())) < 1e-6 * abs(float(fd))
    assert abs(float(L) - float(refocus.loss(u, Hz, t))) < 1e-12 * abs(float(L))
