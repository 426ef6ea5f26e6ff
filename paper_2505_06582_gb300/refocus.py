"""The differentiable workload's loss: refocused intensities of the SLM field (PyTorch).

This is the caller's side of the boundary (the loss a user optimises Gaussians with, as in
the paper's optimisation of the hologram against focal-stack targets): the SLM field u
(from ``gws.gws_field`` / ``gws.forward``) is propagated to focal planes z by the angular
spectrum method (Eq. 3-4: centred DFT, transfer function H(f, +z) = exp(+j 2 pi z f_z) inside
the band and 0 outside, centred inverse DFT), and

    L = sum_z sum_lambda || |u_z|^2 - t_{z,lambda} ||^2.

Its gradient dL/du (PyTorch's complex convention) is what ``gws.backward`` takes.  Everything
here is plain torch; the hologram itself is computed by the library.
"""
from __future__ import annotations

import math

import numpy as np
import torch


def transfer(slm, zs, device, dtype=torch.complex64) -> torch.Tensor:
    """H(f, +z) on the centred grid, [n_lambda][len(zs)][H][W] (0 where f is evanescent)."""
    fx = (np.arange(slm.W) - slm.W // 2) / (slm.W * slm.pitch_x)
    fy = (np.arange(slm.H) - slm.H // 2) / (slm.H * slm.pitch_y)
    FX, FY = np.meshgrid(fx, fy)
    out = []
    for lam in slm.wavelengths:
        k2 = 1.0 / lam ** 2 - FX ** 2 - FY ** 2
        fz = np.sqrt(np.maximum(k2, 0.0))
        out.append([np.where(k2 > 0, np.exp(2j * math.pi * z * fz), 0.0) for z in zs])
    return torch.as_tensor(np.asarray(out), dtype=dtype, device=device)


def refocused_intensity(u: torch.Tensor, Hz: torch.Tensor) -> torch.Tensor:
    """|ASM(u, +z)|^2 for every wavelength and plane: u [L][H][W] -> [L][Z][H][W]."""
    U = torch.fft.fftshift(torch.fft.fft2(torch.fft.ifftshift(u, dim=(-2, -1))), dim=(-2, -1))
    Uz = U[:, None] * Hz
    uz = torch.fft.fftshift(torch.fft.ifft2(torch.fft.ifftshift(Uz, dim=(-2, -1))), dim=(-2, -1))
    return uz.real ** 2 + uz.imag ** 2


def seeded_targets(seed: int, u: torch.Tensor, Hz: torch.Tensor) -> torch.Tensor:
    """Targets t_{z,lambda} ~ U[0, 1] * mean(|u_z|^2) per plane and wavelength (seeded, on the host)."""
    with torch.no_grad():
        mean = refocused_intensity(u, Hz).mean(dim=(-2, -1), keepdim=True)
    rng = np.random.default_rng(seed)
    t = torch.as_tensor(rng.uniform(0.0, 1.0, tuple(Hz.shape)).astype(np.float32), device=u.device)
    return t * mean.to(t.dtype)


def loss(u: torch.Tensor, Hz: torch.Tensor, targets: torch.Tensor) -> torch.Tensor:
    """sum_z sum_lambda || |ASM(u, +z)|^2 - t ||^2."""
    return ((refocused_intensity(u, Hz) - targets) ** 2).sum()


def field_cotangent(u: torch.Tensor, Hz: torch.Tensor, targets: torch.Tensor) -> tuple[torch.Tensor, torch.Tensor]:
    """(L, dL/du) for a field that is not itself a graph leaf (e.g. the output of gws.forward)."""
    with torch.enable_grad():
        x = u.detach().requires_grad_(True)
        L = loss(x, Hz, targets)
        (g,) = torch.autograd.grad(L, x)
    return L.detach(), g
