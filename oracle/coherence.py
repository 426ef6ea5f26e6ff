"""FP64 oracle of partially coherent Gaussian wave splatting (Eq. 14; Sec. 5 "partially coherent
GWS for view-dependent effects" and the supplement's discussion of directional effects).

TEST INFRASTRUCTURE ONLY (tests, smoke check, CPU baseline of the benchmark): the product
path never imports this module.

One time-multiplexed frame t: every Gaussian's spectrum is Eq. 10 with its canonical spectrum
convolved (in frequency) with the angular kernel K_t(f) = Y_l^m(k_hat(f)) e^{j phi_t(f)}, the
translation ramp applied after the convolution, and the Gaussians summed as in Eq. 12 (T = 1):

    u_hat_i(f) = [ G_i * K_t ](f) e^{-j 2 pi f . mu_i},   G_i = Eq. 10 with mu = 0, c = o = 1,

computed through the spatial domain (a convolution of spectra is a product of fields):
g_i = IDFT(G_i) (the Gaussian's field on its own plane, centred at the origin),
w_i = c_i o_i g_i kappa_t, V_i = DFT(w_i), u_hat = sum_i V_i e^{-j 2 pi f . mu_i}, u = IDFT(u_hat).

Readings (listed in the design notes): ordinary frequency throughout; k_hat = lambda (f_x, f_y,
f_z) the unit propagation direction, K_t = 0 where evanescent (and the convolved spectrum is
dropped there); Y_l^m the real spherical harmonic of the front end's convention (Condon-Shortley
phase, index l^2 + l + m); kappa_t(x) = sum_f K_t(f) e^{j 2 pi f . x} / sqrt(sum_f Y^2), so that
E|kappa_t|^2 = 1 (the paper asks the kernel's time-averaged spatial amplitude to be unity);
phi_t(f) = 2 pi u - pi with u the SplitMix64 output number ((t L + l) H + r) W + c + 1 of the
stream seeded with `seed` (top 53 bits / 2^53), r, c the grid indices of f, l the wavelength
index: independent per frame, wavelength and frequency.  DFTs: the oracle's direct centred DFTs.
"""
from __future__ import annotations

import numpy as np

from . import oracle as O
from .holographics import sh_basis

_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed, counter):
    """SplitMix64 (Steele, Lea and Flood, 2014): output number `counter` (>= 1) of the stream
    whose state starts at `seed`, i.e. mix(seed + counter * 0x9E3779B97F4A7C15).  uint64 arrays."""
    with np.errstate(over="ignore"):
        z = np.asarray(seed, dtype=np.uint64) + np.asarray(counter, dtype=np.uint64) * _GAMMA
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        return z ^ (z >> np.uint64(31))


def phases(slm, seed, frame):
    """phi_t(f) in [-pi, pi), float64 [n_lambda][H][W]."""
    L, H, W = slm.n_lambda, slm.H, slm.W
    idx = np.arange(L * H * W, dtype=np.uint64) + np.uint64(frame) * np.uint64(L * H * W)
    u = (splitmix64(np.uint64(seed), idx + np.uint64(1)) >> np.uint64(11)).astype(np.float64) * 2.0 ** -53
    return (2.0 * np.pi * u - np.pi).reshape(L, H, W)


def frequencies(slm, l):
    """(f_x, f_y, f_z, propagating) on the centred grid for wavelength index l."""
    H, W = slm.H, slm.W
    fx = (np.arange(W) - W // 2) / (W * slm.pitch_x)
    fy = (np.arange(H) - H // 2) / (H * slm.pitch_y)
    FX, FY = np.meshgrid(fx, fy)
    k2 = 1.0 / slm.wavelengths[l] ** 2
    rho2 = FX ** 2 + FY ** 2
    prop = rho2 < k2
    FZ = np.sqrt(np.where(prop, k2 - rho2, 0.0))
    return FX, FY, FZ, prop


def angular_kernel(slm, sh_l, sh_m, seed, frame):
    """K_t [n_lambda][H][W] complex and sqrt(sum_f Y^2) [n_lambda]."""
    phi = phases(slm, seed, frame)
    K = np.zeros((slm.n_lambda, slm.H, slm.W), dtype=np.complex128)
    norm = np.zeros(slm.n_lambda)
    k = sh_l * sh_l + sh_l + sh_m
    for l in range(slm.n_lambda):
        FX, FY, FZ, prop = frequencies(slm, l)
        lam = slm.wavelengths[l]
        d = np.stack([FX * lam, FY * lam, FZ * lam], axis=-1).reshape(-1, 3)
        Y = sh_basis(d, sh_l)[:, k].reshape(slm.H, slm.W)
        Y = np.where(prop, Y, 0.0)
        K[l] = Y * np.exp(1j * phi[l])
        norm[l] = np.sqrt(np.sum(Y * Y))
    return K, norm


def kernel_pattern(slm, sh_l, sh_m, seed, frame):
    """kappa_t(x) [n_lambda][H][W]: sum_f K_t(f) e^{j 2 pi f . x} / sqrt(sum_f Y^2)."""
    K, norm = angular_kernel(slm, sh_l, sh_m, seed, frame)
    dfx, dfy = 1.0 / (slm.W * slm.pitch_x), 1.0 / (slm.H * slm.pitch_y)
    return O.idft(K, slm.pitch_x, slm.pitch_y) / (dfx * dfy) / norm[:, None, None]


def spectrum(scene, slm, sh_l, sh_m, seed, frame, phase_match=False, kappa=None):
    """u_hat_SLM(f) of one frame, complex128 [n_lambda][H][W]; kappa overrides the kernel pattern."""
    px, py = slm.pitch_x, slm.pitch_y
    dfx, dfy = 1.0 / (slm.W * px), 1.0 / (slm.H * py)
    if kappa is None:
        kappa = kernel_pattern(slm, sh_l, sh_m, seed, frame)
    L = slm.n_lambda
    acc = np.zeros((L, slm.H, slm.W), dtype=np.complex128)
    ramps = []
    for l in range(L):
        FX, FY, FZ, prop = frequencies(slm, l)
        ramps.append((FX, FY, FZ, prop))
    for i in range(scene.n):
        one = type(scene)(np.zeros((1, 3)), scene.quat[i:i + 1], scene.scale[i:i + 1],
                          np.ones(1, dtype=np.float32), np.ones((1, L), dtype=np.float32))
        G = O.spectrum(one, slm)                         # Eq. 10 at the origin, on its own plane
        g = O.idft(G, px, py)                            # its field
        w = float(scene.opacity[i]) * scene.amp[i].astype(np.float64)[:, None, None] * g * kappa
        V = O.idft_adjoint(w, px, py) * (px * py) / (dfx * dfy)  # forward DFT x px py
        mu = scene.mean[i].astype(np.float64)
        for l in range(L):
            FX, FY, FZ, prop = ramps[l]
            ph = -2.0 * np.pi * (FX * mu[0] + FY * mu[1] + FZ * mu[2])
            if phase_match:
                ph = ph + 2.0 * np.pi * mu[2] / slm.wavelengths[l]
            acc[l] += np.where(prop, V[l] * np.exp(1j * ph), 0.0)
    return acc


def field(scene, slm, sh_l, sh_m, seed, frame, phase_match=False, kappa=None):
    """u_SLM of one frame: the centred inverse DFT (Eq. 3) of `spectrum`."""
    return O.idft(spectrum(scene, slm, sh_l, sh_m, seed, frame, phase_match, kappa), slm.pitch_x, slm.pitch_y)


def expected_power(scene_one, slm, sh_l, sh_m):
    """E_phi |V(f)|^2 for one Gaussian at the origin: (1 / sum Y^2) sum_f' Y(f')^2 |G(f - f')|^2
    (circular convolution on the grid), computed in the frequency domain."""
    L = slm.n_lambda
    K, norm = angular_kernel(slm, sh_l, sh_m, 0, 0)
    G = O.spectrum(scene_one, slm)
    out = np.zeros((L, slm.H, slm.W))
    for l in range(L):
        Y2 = np.abs(K[l]) ** 2
        P = np.abs(G[l]) ** 2
        # circular convolution through the FFT (a library step): centred grids share the origin
        conv = np.real(np.fft.ifft2(np.fft.fft2(np.fft.ifftshift(Y2)) * np.fft.fft2(np.fft.ifftshift(P))))
        out[l] = np.fft.fftshift(conv) / norm[l] ** 2
    return out
