"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: a brute-force
numerical Fourier transform, closed forms, Parseval, invariances, hand-derived
transmittances, finite differences and library routines (numpy FFT, stable argsort).
A plausible mistake in the oracle (a dropped term, a wrong sign, a transposed operand,
a wrong constant) fails at least one of them.
"""
import math

import numpy as np
import pytest

import oracle as O
from paper_2505_06582_gb300.scenes import SLM, uniform_scene, random_field
from tests.helpers import grid_freqs, make_scene, qaxis, qmul, rel_l2, rotmat

LAM = 520e-9
SLM_SMALL = SLM(48, 64, 8e-6, 6e-6, (LAM,))  # non-square grid, different pitches in x and y


def _periodised_sample(fn, xs, ys, period_x, period_y, images=2):
    """Sum of the images of fn over (2 images + 1)^2 periods, sampled on the xs, ys grid."""
    X, Y = np.meshgrid(xs, ys)
    out = np.zeros_like(X)
    for kx in range(-images, images + 1):
        for ky in range(-images, images + 1):
            out += fn(X + kx * period_x, Y + ky * period_y)
    return out


def _brute_force_plane_spectrum(a_fn, slm: SLM, oversample=16):
    """Continuous FT of a plane field a(x, y) at the SLM grid frequencies.

    The field is sampled (periodised over the SLM aperture) on a grid `oversample` times
    finer than the SLM pitch; dx dy * DFT of one period equals the Fourier-series
    coefficients, i.e. the FT sampled at k / aperture (Poisson summation).  The central
    H x W bins have the SLM grid's frequencies."""
    Ny, Nx = slm.H * oversample, slm.W * oversample
    dx, dy = slm.pitch_x / oversample, slm.pitch_y / oversample
    xs = (np.arange(Nx) - Nx // 2) * dx
    ys = (np.arange(Ny) - Ny // 2) * dy
    a = _periodised_sample(a_fn, xs, ys, Nx * dx, Ny * dy)
    A = dx * dy * np.fft.fftshift(np.fft.fft2(np.fft.ifftshift(a)))
    r0, c0 = Ny // 2 - slm.H // 2, Nx // 2 - slm.W // 2
    return A[r0:r0 + slm.H, c0:c0 + slm.W]


def _gauss2d(mu_xy, S2inv):
    def fn(X, Y):
        dx, dy = X - mu_xy[0], Y - mu_xy[1]
        return np.exp(-0.5 * (S2inv[0, 0] * dx * dx + 2 * S2inv[0, 1] * dx * dy + S2inv[1, 1] * dy * dy))
    return fn


# ---------------------------------------------------------------------------------------
# T1: brute force
# ---------------------------------------------------------------------------------------

def test_t1_untilted_matches_brute_force_fft():
    """Untilted Gaussians (in-plane rotation only): FFT of the 16x oversampled plane field,
    times the angular-spectrum propagator H(f, -z), equals the closed form (Eq. 10, Eq. 12)."""
    rng = np.random.default_rng(11)
    slm = SLM_SMALL
    FX, FY, FZ = grid_freqs(slm, LAM)
    total_bf = np.zeros((slm.H, slm.W), complex)
    means, quats, scales, opas, amps = [], [], [], [], []
    for k in range(3):
        psi = rng.uniform(0, 2 * math.pi)
        q = qaxis([0, 0, 1], psi)
        su, sv = rng.uniform(2.0, 3.5) * slm.pitch_x, rng.uniform(2.0, 3.5) * slm.pitch_y
        mu = np.array([rng.uniform(-100e-6, 100e-6), rng.uniform(-60e-6, 60e-6), rng.uniform(1e-3, 5e-3)])
        o, c = rng.uniform(0.2, 1.0), rng.uniform(0.2, 1.0)
        R2 = rotmat(q)[:2, :2]
        Sig = R2 @ np.diag([su * su, sv * sv]) @ R2.T
        A = _brute_force_plane_spectrum(_gauss2d(mu[:2], np.linalg.inv(Sig)), slm)
        total_bf += c * o * A * np.exp(-2j * math.pi * FZ * mu[2])
        means.append(mu); quats.append(q); scales.append([su, sv]); opas.append(o); amps.append([c])
    sc = make_scene(means, quats, scales, opas, amps)
    U = O.spectrum(sc, slm)[0]
    assert rel_l2(U, total_bf) < 1e-10


def test_t1_tilted_matches_local_plane_quadrature():
    """Tilted Gaussian: direct quadrature of the Gaussian on its own plane, illuminated by
    the on-axis plane wave (local phase ramp from f_r), evaluated at the remapped local
    frequencies, times the numerically differentiated Jacobian of the frequency remap and
    the translation / propagation phase -- equals the closed form."""
    slm = SLM(24, 32, 8e-6, 8e-6, (LAM,))
    q = qmul(qaxis([1, 0.3, 0], math.radians(35)), qaxis([0, 0, 1], 0.7))
    R = rotmat(q)
    r1, r2 = R[:, 0], R[:, 1]
    su, sv = 2.2 * 8e-6, 3.1 * 8e-6
    mu = np.array([20e-6, -15e-6, 2.5e-3])
    sc = make_scene([mu], [q], [[su, sv]], [0.9], [[0.7]])
    U = O.spectrum(sc, slm)[0]

    FX, FY, FZ = grid_freqs(slm, LAM)
    fr = np.array([0, 0, 1 / LAM])

    def local_freq(fx, fy):
        fz = np.sqrt(1 / LAM ** 2 - fx ** 2 - fy ** 2)
        f = np.stack([fx, fy, fz], -1)
        return (f - fr) @ r1, (f - fr) @ r2, f @ r1, f @ r2

    nu_u, nu_v, _, _ = local_freq(FX, FY)
    # 1D quadratures (the local Gaussian is separable in its own axes)
    def quad1d(s, nu):
        x = np.arange(-12 * 8, 12 * 8 + 1) * (s / 8)
        w = np.exp(-0.5 * (x / s) ** 2) * (s / 8)
        return np.tensordot(np.exp(-2j * math.pi * nu[..., None] * x), w, axes=([-1], [0]))
    local = quad1d(su, nu_u) * quad1d(sv, nu_v)
    # Jacobian |det d(alpha, beta)/d(fx, fy)| of the remap (alpha, beta) = (r1.f, r2.f)
    h = 1e-3 / (slm.W * slm.pitch_x)
    _, _, ap, bp = local_freq(FX + h, FY)
    _, _, am, bm = local_freq(FX - h, FY)
    _, _, aq, bq = local_freq(FX, FY + h)
    _, _, an, bn = local_freq(FX, FY - h)
    J = np.abs(((ap - am) * (bq - bn) - (aq - an) * (bp - bm)) / (4 * h * h))
    bf = 0.9 * 0.7 * J * local * np.exp(-2j * math.pi * (FX * mu[0] + FY * mu[1] + FZ * mu[2]))
    assert rel_l2(U, bf) < 1e-7


# ---------------------------------------------------------------------------------------
# T2: analytic untilted fields
# ---------------------------------------------------------------------------------------

def test_t2_in_focus_field_is_the_sampled_gaussian():
    """mu_z = 0, untilted, s >= 3 px: the field (centred inverse DFT x dfx dfy) equals the
    periodised Gaussian c o exp(-1/2 |S^-1 R^T (x - mu)|^2) at the pixel centres."""
    slm = SLM(64, 80, 8e-6, 8e-6, (LAM,))
    q = qaxis([0, 0, 1], 0.4)
    su, sv = 3.2 * 8e-6, 4.5 * 8e-6
    mu = np.array([40e-6, -24e-6, 0.0])  # on a pixel centre
    sc = make_scene([mu], [q], [[su, sv]], [0.8], [[0.6]])
    u = O.field(sc, slm)[0]
    R2 = rotmat(q)[:2, :2]
    Sig = R2 @ np.diag([su * su, sv * sv]) @ R2.T
    xs = (np.arange(slm.W) - slm.W // 2) * slm.pitch_x
    ys = (np.arange(slm.H) - slm.H // 2) * slm.pitch_y
    ref = 0.48 * _periodised_sample(_gauss2d(mu[:2], np.linalg.inv(Sig)), xs, ys, slm.W * slm.pitch_x,
                                    slm.H * slm.pitch_y)
    assert np.abs(u - ref).max() < 1e-11
    assert abs(np.abs(u).max() - 0.48) < 1e-12  # peak c o at the centre


def test_t2_fresnel_gaussian_beam():
    """An untilted isotropic Gaussian at depth z: the spectrum agrees with the paraxial
    (Fresnel) Gaussian-beam closed form 2 pi s^2 exp(-2 pi^2 s^2 f^2) exp(-j 2 pi z / lam)
    exp(+j pi lam z f^2) exp(-j 2 pi f.mu_xy); the remaining difference is the
    non-paraxial phase 2 pi z (lam^3 f^4 / 8 + ...), bounded here by 1e-5."""
    slm = SLM(64, 64, 8e-6, 8e-6, (LAM,))
    s, z = 4 * 8e-6, 2e-3
    mu = np.array([10e-6, -30e-6, z])
    sc = make_scene([mu], [[1, 0, 0, 0]], [[s, s]], [1.0], [[1.0]])
    U = O.spectrum(sc, slm)[0]
    FX, FY, _ = grid_freqs(slm, LAM)
    F2 = FX ** 2 + FY ** 2
    par = (2 * math.pi * s * s * np.exp(-2 * math.pi ** 2 * s * s * F2) * np.exp(-2j * math.pi * z / LAM)
           * np.exp(1j * math.pi * LAM * z * F2) * np.exp(-2j * math.pi * (FX * mu[0] + FY * mu[1])))
    err = rel_l2(U, par)
    assert err < 1e-5
    # the bound is not vacuous: the paraxial phase itself is large over the band
    assert np.abs(np.angle(np.exp(1j * math.pi * LAM * z * F2))).max() > 1.0


def test_t2_refocus_identity():
    """Propagating the SLM field forward by +mu_z (H(f, +z) = exp(+j 2 pi z fz)) gives the
    in-focus (mu_z = 0) field: the sign convention of Eq. 5 / Eq. 12 (propagation by -z_i)."""
    slm = SLM_SMALL
    rng = np.random.default_rng(3)
    q = rng.normal(size=4)
    mu = np.array([5e-6, 7e-6, 3.3e-3])
    sc = make_scene([mu], [q], [[20e-6, 14e-6]], [0.7], [[0.9]])
    sc0 = make_scene([[mu[0], mu[1], 0.0]], [q], [[20e-6, 14e-6]], [0.7], [[0.9]])
    _, _, FZ = grid_freqs(slm, LAM)
    U = O.spectrum(sc, slm)[0] * np.exp(2j * math.pi * FZ * mu[2])
    U0 = O.spectrum(sc0, slm)[0]
    assert rel_l2(U, U0) < 1e-11


# ---------------------------------------------------------------------------------------
# T3 Parseval, T4 order invariance, T5 projected limit
# ---------------------------------------------------------------------------------------

def test_t3_parseval_discrete_and_continuous():
    slm = SLM(40, 56, 8e-6, 6e-6, (LAM, 638e-9))
    sc = uniform_scene(5, 12, slm, scale_median_px=3.0)
    U = O.spectrum(sc, slm)
    u = O.idft(U, slm.pitch_x, slm.pitch_y)
    dfx, dfy = 1 / (slm.W * slm.pitch_x), 1 / (slm.H * slm.pitch_y)
    for l in range(2):
        e_space = (np.abs(u[l]) ** 2).sum() * slm.pitch_x * slm.pitch_y
        e_freq = (np.abs(U[l]) ** 2).sum() * dfx * dfy
        assert abs(e_space - e_freq) < 1e-12 * e_freq
    # one untilted in-band Gaussian: energy pi s_u s_v (c o)^2, independent of its depth
    # (aperture >= 12 sigma so that the periodic images do not overlap)
    slm = SLM(72, 80, 8e-6, 6e-6, (LAM, 638e-9))
    dfx, dfy = 1 / (slm.W * slm.pitch_x), 1 / (slm.H * slm.pitch_y)
    for z in (0.0, 4e-3):
        g = make_scene([[0, 0, z]], [qaxis([0, 0, 1], 0.3)], [[3.5 * 8e-6, 5 * 6e-6]], [0.6], [[0.5, 0.5]])
        Ug = O.spectrum(g, slm)
        e = (np.abs(Ug[0]) ** 2).sum() * dfx * dfy
        assert abs(e - math.pi * 3.5 * 8e-6 * 5 * 6e-6 * 0.09) < 1e-9 * e


def test_t4_order_invariance():
    slm = SLM_SMALL
    sc = uniform_scene(7, 20, slm)
    perm = np.random.default_rng(1).permutation(sc.n)
    U = O.spectrum(sc, slm)
    Up = O.spectrum(sc.subset(perm), slm)
    assert rel_l2(Up, U) < 1e-14


def test_t5_projected_footprint_limit():
    """For lam -> 0 the spectrum tends to the FT of the Gaussian projected along z,
    2 pi |det M| exp(-2 pi^2 f^T M M^T f), times the propagator: this fixes the reference
    wave shift f_r and the Jacobian |n_z| (without the shift the tilted Gaussian vanishes)."""
    lam = 1e-10
    slm = SLM(48, 48, 8e-6, 8e-6, (lam,))
    q = qmul(qaxis([0.2, 1, 0], math.radians(50)), qaxis([0, 0, 1], 1.1))
    R = rotmat(q)
    su, sv = 3 * 8e-6, 2 * 8e-6
    mu = np.array([12e-6, -9e-6, 1.5e-3])
    sc = make_scene([mu], [q], [[su, sv]], [1.0], [[1.0]])
    U = O.spectrum(sc, slm)[0]
    M = np.stack([su * R[:2, 0], sv * R[:2, 1]], 1)
    A = _brute_force_plane_spectrum(_gauss2d(mu[:2], np.linalg.inv(M @ M.T)), slm)
    _, _, FZ = grid_freqs(slm, lam)
    ref = A * np.exp(-2j * math.pi * FZ * mu[2])
    assert rel_l2(U, ref) < 2e-5
    # and the peak at f = 0 is 2 pi s_u s_v |n_z|
    assert abs(abs(U[24, 24]) - 2 * math.pi * su * sv * abs(R[2, 2])) < 1e-6 * abs(U[24, 24])


# ---------------------------------------------------------------------------------------
# T6 invariances, T7 periodicity, T8 linearity
# ---------------------------------------------------------------------------------------

def test_t6_invariances():
    slm = SLM_SMALL
    rng = np.random.default_rng(9)
    q = rng.normal(size=4)
    mu = [14e-6, -3e-6, 2e-3]
    base = O.spectrum(make_scene([mu], [q], [[17e-6, 11e-6]], [0.5], [[0.8]]), slm)
    neg = O.spectrum(make_scene([mu], [-q], [[17e-6, 11e-6]], [0.5], [[0.8]]), slm)
    flip = O.spectrum(make_scene([mu], [qmul(q, [0, 1, 0, 0])], [[17e-6, 11e-6]], [0.5], [[0.8]]), slm)
    swap = O.spectrum(make_scene([mu], [qmul(q, qaxis([0, 0, 1], math.pi / 2))], [[11e-6, 17e-6]], [0.5], [[0.8]]),
                      slm)
    assert rel_l2(neg, base) < 1e-13
    assert rel_l2(flip, base) < 1e-13
    assert rel_l2(swap, base) < 1e-13
    # scaling the quaternion changes nothing (it is normalised)
    big = O.spectrum(make_scene([mu], [3.7 * q], [[17e-6, 11e-6]], [0.5], [[0.8]]), slm)
    assert rel_l2(big, base) < 1e-13


def test_t7_periodicity():
    slm = SLM_SMALL
    sc = uniform_scene(2, 6, slm)
    sh = sc.subset(np.arange(sc.n))
    sh.mean[:, 0] += slm.W * slm.pitch_x
    sh.mean[:, 1] -= 2 * slm.H * slm.pitch_y
    assert rel_l2(O.spectrum(sh, slm), O.spectrum(sc, slm)) < 1e-11


@pytest.mark.parametrize("blend", [O.BLEND_OIT, O.BLEND_SORTED_T])
def test_t8_linearity_for_separated_groups(blend):
    slm = SLM(48, 96, 8e-6, 8e-6, (LAM,))
    a = uniform_scene(21, 5, slm, scale_median_px=1.5, sigma_log=0.1)
    b = uniform_scene(22, 5, slm, scale_median_px=1.5, sigma_log=0.1)
    a.mean[:, 0] = -200e-6 + 0.2 * a.mean[:, 0]
    b.mean[:, 0] = 200e-6 + 0.2 * b.mean[:, 0]
    ab = a.concat(b)
    Ua, Ub, Uab = (O.spectrum(s, slm, blend=blend) for s in (a, b, ab))
    assert rel_l2(Uab, Ua + Ub) < 1e-13


# ---------------------------------------------------------------------------------------
# T9-T11 occlusion with the depth-sorted transmittance
# ---------------------------------------------------------------------------------------

def test_t9_full_occlusion_behind_opaque_front():
    slm = SLM_SMALL
    front = make_scene([[0, 0, 2e-3]], [[1, 0, 0, 0]], [[80e-6, 60e-6]], [1.0], [[0.7]])
    rear = make_scene([[0, 0, 4e-3]], [qaxis([1, 0, 0], 0.5)], [[20e-6, 20e-6]], [0.8], [[0.9]])
    both = rear.concat(front)  # input order is not depth order
    T = O.transmittance(both)
    assert T[1] == 1.0 and T[0] == 0.0
    Us = O.spectrum(both, slm, blend=O.BLEND_SORTED_T)
    Uf = O.spectrum(front, slm)
    assert np.array_equal(Us, Uf)
    # the order-invariant sum does not occlude: front + rear
    Uo = O.spectrum(both, slm, blend=O.BLEND_OIT)
    assert rel_l2(Uo, Uf + O.spectrum(rear, slm)) < 1e-14


def test_t10_limits():
    slm = SLM_SMALL
    one = uniform_scene(4, 1, slm)
    assert np.array_equal(O.spectrum(one, slm, blend=O.BLEND_SORTED_T), O.spectrum(one, slm))
    sc = uniform_scene(4, 10, slm)
    sc.opacity[:] = 0.0
    assert np.array_equal(O.transmittance(sc), np.ones(10))


def test_t11_two_gaussian_hand_cases():
    s1, o1, d = 24e-6, 0.7, 1.5 * 24e-6
    sc = make_scene([[0, 0, 2e-3], [d, 0, 3e-3]], [[1, 0, 0, 0], [1, 0, 0, 0]], [[s1, s1], [9e-6, 9e-6]],
                    [o1, 0.5], [[1.0], [1.0]])
    T = O.transmittance(sc)
    assert T[0] == 1.0
    assert abs(T[1] - (1 - o1 * math.exp(-0.5 * 1.5 ** 2))) < 1e-15
    # anisotropic, rotated front Gaussian: alpha = o exp(-1/2 (dx'^2/su^2 + dy'^2/sv^2)) in its axes
    psi = 0.6
    su, sv = 30e-6, 12e-6
    dx, dy = 10e-6, 7e-6
    xr = math.cos(psi) * dx + math.sin(psi) * dy
    yr = -math.sin(psi) * dx + math.cos(psi) * dy
    sc = make_scene([[0, 0, 2e-3], [dx, dy, 5e-3]], [qaxis([0, 0, 1], psi), [1, 0, 0, 0]], [[su, sv], [9e-6, 9e-6]],
                    [0.9, 0.5], [[1.0], [1.0]])
    assert abs(O.transmittance(sc)[1] - (1 - 0.9 * math.exp(-0.5 * (xr ** 2 / su ** 2 + yr ** 2 / sv ** 2)))) < 1e-15
    # tilted front Gaussian: the footprint is the projection, foreshortened by cos(tilt) along y
    tilt = 0.8
    sc = make_scene([[0, 0, 2e-3], [0, 12e-6, 5e-3]], [qaxis([1, 0, 0], tilt), [1, 0, 0, 0]],
                    [[20e-6, 20e-6], [9e-6, 9e-6]], [0.9, 0.5], [[1.0], [1.0]])
    sy = 20e-6 * math.cos(tilt)
    assert abs(O.transmittance(sc)[1] - (1 - 0.9 * math.exp(-0.5 * (12e-6 / sy) ** 2))) < 1e-14
    # below t_eps = 1/255 the front Gaussian is ignored
    far = math.sqrt(2 * math.log(0.7 * 255 / 0.9)) * s1  # alpha = 0.9/255 < 1/255
    sc = make_scene([[0, 0, 2e-3], [far, 0, 3e-3]], [[1, 0, 0, 0]] * 2, [[s1, s1]] * 2, [o1, 0.5], [[1.0], [1.0]])
    assert O.transmittance(sc)[1] == 1.0
    # just above t_eps the front Gaussian counts: alpha = 1.2/255
    near = math.sqrt(2 * math.log(0.7 * 255 / 1.2)) * s1
    sc = make_scene([[0, 0, 2e-3], [near, 0, 3e-3]], [[1, 0, 0, 0]] * 2, [[s1, s1]] * 2, [o1, 0.5], [[1.0], [1.0]])
    assert abs(O.transmittance(sc)[1] - (1 - 1.2 / 255)) < 1e-15
    # equal depths: the lower input index is in front
    sc = make_scene([[0, 0, 3e-3], [0, 0, 3e-3]], [[1, 0, 0, 0]] * 2, [[s1, s1]] * 2, [0.4, 0.5], [[1.0], [1.0]])
    T = O.transmittance(sc)
    assert T[0] == 1.0 and abs(T[1] - 0.6) < 1e-15


# ---------------------------------------------------------------------------------------
# DFT, sort and DPAC pins
# ---------------------------------------------------------------------------------------

@pytest.mark.parametrize("H,W", [(8, 12), (7, 10), (9, 5), (1, 6)])
def test_idft_matches_numpy_and_its_adjoint(H, W):
    px, py = 8e-6, 5e-6
    x = random_field(1, (H, W))
    y = random_field(2, (H, W))
    u = O.idft(x, px, py)
    ref = (1 / (W * px)) * (1 / (H * py)) * H * W * np.fft.fftshift(np.fft.ifft2(np.fft.ifftshift(x)))
    assert rel_l2(u, ref) < 1e-13
    # <A x, y> = <x, A^H y>
    lhs = np.vdot(y, u)
    rhs = np.vdot(O.idft_adjoint(y, px, py), x)
    assert abs(lhs - rhs) < 1e-12 * abs(lhs)
    at = O.idft_at(x, px, py, [0, H - 1, H // 2], [W - 1, 0, W // 2])
    assert np.allclose(at, [u[0, W - 1], u[H - 1, 0], u[H // 2, W // 2]], rtol=1e-12, atol=0)


def test_depth_order_is_the_stable_argsort():
    rng = np.random.default_rng(0)
    mean = rng.normal(size=(500, 3))
    mean[::7, 2] = 0.25  # ties
    mean[3, 2] = -0.0
    mean[4, 2] = 0.0
    assert np.array_equal(O.depth_order(mean), np.argsort(mean[:, 2], kind="stable"))


def test_dpac_identity_and_checkerboard():
    f = random_field(5, (2, 6, 7), zero_frac=0.1)
    P = O.encode(f)
    assert P.min() >= -math.pi and P.max() < math.pi
    for l in range(2):
        amax = np.abs(f[l]).max()
        a = np.abs(f[l]) / amax
        phi = np.angle(f[l])
        r, c = np.meshgrid(np.arange(6), np.arange(7), indexing="ij")
        even = (r + c) % 2 == 0
        d = P[l] - phi
        # double-phase: e^{jP} = e^{j phi} (a -/+ j sqrt(1 - a^2)): cos(P - phi) = a, sign of sin by parity
        assert np.allclose(np.cos(d), a, atol=1e-12)
        s = np.sin(d)
        assert np.all(s[even] <= 1e-12) and np.all(s[~even] >= -1e-12)
        # the mean of the two phasors rebuilds a e^{j phi}
        p1 = phi - np.arccos(np.clip(a, 0, 1))
        p2 = phi + np.arccos(np.clip(a, 0, 1))
        assert np.allclose(0.5 * (np.exp(1j * p1) + np.exp(1j * p2)), a * np.exp(1j * phi), atol=1e-12)
    # a fixed amplitude scale clamps above it
    P2 = O.encode(f, amp_scale=float(np.abs(f).max()) / 4)
    assert np.isfinite(P2).all()


# ---------------------------------------------------------------------------------------
# T13: gradients
# ---------------------------------------------------------------------------------------

def _loss(scene, slm, G, blend):
    U = O.spectrum(scene, slm, blend=blend)
    return float(np.real(np.vdot(G, U)))  # sum Re(conj(G) U)


def _fd_grad(scene, slm, G, blend, field, idx, h):
    sp = scene.subset(np.arange(scene.n))
    sm = scene.subset(np.arange(scene.n))
    getattr(sp, field)[idx] += h
    getattr(sm, field)[idx] -= h
    return (_loss(sp, slm, G, blend) - _loss(sm, slm, G, blend)) / (2 * h)


@pytest.mark.parametrize("blend", [O.BLEND_OIT, O.BLEND_SORTED_T])
def test_t13_gradients_match_central_differences(blend):
    slm = SLM(20, 24, 8e-6, 8e-6, (638e-9, 450e-9))
    if blend == O.BLEND_OIT:
        u = uniform_scene(13, 4, slm, scale_median_px=2.0)
        sc = make_scene(u.mean, u.quat, u.scale, u.opacity, u.amp)  # float64 copy for the differences
    else:
        # overlapping footprints with alphas well away from 1/255
        sc = make_scene([[0, 0, 2e-3], [12e-6, -6e-6, 3e-3], [-8e-6, 10e-6, 4e-3]],
                        [qaxis([1, 0.4, 0], 0.5), qaxis([0.3, 1, 0], 0.4), qaxis([0, 0, 1], 1.0)],
                        [[25e-6, 18e-6], [20e-6, 22e-6], [15e-6, 17e-6]], [0.8, 0.6, 0.7],
                        [[0.9, 0.4], [0.5, 0.8], [0.7, 0.6]])
        T = O.transmittance(sc)
        assert T[1] < 0.9 and T[2] < 0.9
    G = random_field(4, (slm.n_lambda, slm.H, slm.W)) * 1e8
    g = O.backward_spectrum(sc, slm, G, blend=blend)
    for field, scale in (("mean", 1e-5), ("quat", 1.0), ("scale", 1e-5), ("opacity", 1.0), ("amp", 1.0)):
        arr = getattr(sc, field)
        fd = np.zeros_like(arr)
        for idx in np.ndindex(arr.shape):
            # the mean enters through the phase 2 pi f.mu with f_z ~ 2e6 /m: a 1e-11 m step keeps
            # the central-difference truncation error (h 2 pi f_z)^2 / 6 below 1e-8
            h = 1e-11 if field == "mean" else 1e-6 * (abs(arr[idx]) + scale)
            fd[idx] = _fd_grad(sc, slm, G, blend, field, idx, h)
        assert rel_l2(g[field], fd) < 1e-6, field


def test_t13_gradients_agree_with_torch_autograd_restatement():
    """Third opinion: a dense FP64 torch restatement of the spectrum (test-only code),
    differentiated by autograd, including PyTorch's complex-gradient convention."""
    torch = pytest.importorskip("torch")
    slm = SLM(16, 20, 8e-6, 8e-6, (520e-9, 450e-9))
    sc = uniform_scene(31, 3, slm, scale_median_px=2.0)
    G = random_field(8, (slm.n_lambda, slm.H, slm.W))
    g = O.backward_field(sc, slm, G)

    t = {k: torch.tensor(getattr(sc, k), dtype=torch.float64, requires_grad=True)
         for k in ("mean", "quat", "scale", "opacity", "amp")}
    q = t["quat"] / t["quat"].norm(dim=1, keepdim=True)
    w, x, y, z = q.unbind(1)
    r1 = torch.stack([1 - 2 * (y * y + z * z), 2 * (x * y + w * z), 2 * (x * z - w * y)], 1)
    r2 = torch.stack([2 * (x * y - w * z), 1 - 2 * (x * x + z * z), 2 * (y * z + w * x)], 1)
    r3 = torch.stack([2 * (x * z + w * y), 2 * (y * z - w * x), 1 - 2 * (x * x + y * y)], 1)
    fields = []
    for l, lam in enumerate(slm.wavelengths):
        FX, FY, FZ = (torch.tensor(a) for a in grid_freqs(slm, lam))
        f = torch.stack([FX, FY, FZ], -1)[None]  # 1,H,W,3
        d = f - torch.tensor([0, 0, 1 / lam], dtype=torch.float64)
        a = (d * r1[:, None, None]).sum(-1)
        b = (d * r2[:, None, None]).sum(-1)
        gg = (f * r3[:, None, None]).sum(-1)
        su, sv = t["scale"][:, 0, None, None], t["scale"][:, 1, None, None]
        amp = 2 * math.pi * su * sv * gg.abs() / FZ * torch.exp(-2 * math.pi ** 2 * (su ** 2 * a ** 2 + sv ** 2 * b ** 2))
        cyc = -(f * t["mean"][:, None, None]).sum(-1)
        term = amp * torch.exp(2j * math.pi * cyc)
        wgt = (t["amp"][:, l] * t["opacity"])[:, None, None]
        U = (wgt * term).sum(0)
        dfx, dfy = 1 / (slm.W * slm.pitch_x), 1 / (slm.H * slm.pitch_y)
        u = dfx * dfy * slm.H * slm.W * torch.fft.fftshift(torch.fft.ifft2(torch.fft.ifftshift(U)))
        fields.append(u)
    u = torch.stack(fields)
    Gt = torch.tensor(G)
    L = (Gt.conj() * u).real.sum()
    L.backward()
    for k in t:
        assert rel_l2(g[k], t[k].grad.numpy()) < 1e-9, k


def test_subset_backward_equals_full_backward():
    slm = SLM(18, 22, 8e-6, 8e-6, (638e-9, 450e-9))
    sc = uniform_scene(41, 6, slm, scale_median_px=2.0)
    G = random_field(6, (2, 18, 22))
    full = O.backward_spectrum(sc, slm, G)
    sub = O.backward_spectrum_at(sc, slm, G, [4, 1])
    for k in full:
        assert np.allclose(sub[k], full[k][[4, 1]], rtol=1e-13, atol=0), k


# ---------------------------------------------------------------------------------------
# exact alpha wave blending (Algorithm S2)
# ---------------------------------------------------------------------------------------

def test_exact_awb_without_occlusion_is_the_order_invariant_sum():
    """alpha below t_eps everywhere -> T = 1 -> F(F^-1(u_k)) H(f, -z_k) sums to Eq. 12 exactly:
    pins the DFT scales and the propagation sign against the independently pinned closed form."""
    slm = SLM(24, 32, 8e-6, 6e-6, (638e-9, 450e-9))
    sc = uniform_scene(61, 7, slm, scale_median_px=2.5)
    sc.opacity[:] = 0.9 / 255
    assert np.abs(O.exact_awb(sc, slm) - O.spectrum(sc, slm)).max() < 1e-10 * np.abs(O.spectrum(sc, slm)).max()
    one = sc.subset([3])
    one.opacity[:] = 0.8
    assert rel_l2(O.exact_awb(one, slm), O.spectrum(one, slm)) < 1e-11


def test_exact_awb_transmittance_map_by_hand():
    """Untilted in-focus Gaussians (|u_k| = G_k on the grid): T = prod (1 - o_k G_k) where o_k G_k > t_eps."""
    slm = SLM(48, 48, 8e-6, 8e-6, (520e-9,))
    s1, s2 = 4 * 8e-6, 3 * 8e-6
    sc = make_scene([[0, 0, 1e-3], [24e-6, -16e-6, 3e-3]], [[1, 0, 0, 0]] * 2, [[s1, s1], [s2, s2]], [0.7, 0.5],
                    [[1.0], [1.0]])
    _, T = O.exact_awb(sc, slm, with_T=True)
    xs = (np.arange(48) - 24) * 8e-6
    X, Y = np.meshgrid(xs, xs)
    a1 = 0.7 * np.exp(-0.5 * (X ** 2 + Y ** 2) / s1 ** 2)
    a2 = 0.5 * np.exp(-0.5 * ((X - 24e-6) ** 2 + (Y + 16e-6) ** 2) / s2 ** 2)
    ref = (1 - np.where(a1 > 1 / 255, a1, 0)) * (1 - np.where(a2 > 1 / 255, a2, 0))
    assert np.abs(T[0] - ref).max() < 1e-9


def test_exact_awb_binarized_disk_hides_what_is_behind():
    """t_binarize (disk occlusion): an opaque disk in front of a small Gaussian hides it."""
    # the rear Gaussian (2.5 px) is band-limited on this grid only by e^-31, so its field has
    # no ringing outside the disk (|u_front| > 0.05 within ~29 px of the front's centre)
    slm = SLM(80, 80, 8e-6, 8e-6, (520e-9,))
    front = make_scene([[0, 0, 2e-3]], [[1, 0, 0, 0]], [[12 * 8e-6, 12 * 8e-6]], [1.0], [[0.6]])
    rear = make_scene([[8e-6, 0, 5e-3]], [[1, 0, 0, 0]], [[2.5 * 8e-6, 2.5 * 8e-6]], [0.9], [[0.8]])
    both = rear.concat(front)
    got = O.exact_awb(both, slm, binarize=0.05)
    only_front = O.exact_awb(front, slm, binarize=0.05)
    assert rel_l2(got, only_front) < 1e-9
    # without the disk the rear Gaussian shows through (soft alpha)
    assert rel_l2(O.exact_awb(both, slm), only_front) > 1e-3


# ---------------------------------------------------------------------------------------
# phase matching (Sec. 4.1 reference wave; supplement, hardware setup: each wavefront's
# phase matched) and the per-pixel Gaussian exponent
# ---------------------------------------------------------------------------------------

def _phase_match_scene():
    """Five Gaussians: untilted and tilted, off-axis, at three depths."""
    return make_scene([[0, 0, 1.3e-3], [40e-6, -24e-6, 2.77e-3], [-56e-6, 8e-6, 4.1e-3], [16e-6, 30e-6, 2.77e-3],
                       [-8e-6, -40e-6, 1.3e-3]],
                      [[1, 0, 0, 0], qaxis([0, 0, 1], 0.7), qaxis([1, 0.3, 0], 0.5), qaxis([0.2, 1, 0], 0.9),
                       qaxis([1, 1, 0.5], 1.2)],
                      [[20e-6, 14e-6], [16e-6, 24e-6], [18e-6, 12e-6], [22e-6, 19e-6], [15e-6, 15e-6]],
                      [0.9, 0.5, 0.7, 0.35, 0.8], [[0.6, 0.4], [0.9, 0.2], [0.3, 0.8], [0.5, 0.5], [0.7, 0.1]])


def test_phase_match_dc_value_is_real_and_the_closed_form():
    """With phase matching the on-axis plane wave f = 0 (f_z = 1/lam, d = f - f_r = 0) carries no
    phase: every Gaussian's DC value is real and positive, W 2 pi s_u s_v |r3_z| (Eq. 10 at f = 0:
    |r3.f| / f_z = |r3_z|, exp(0) = 1), whatever its depth and lateral position.  Without it the same
    value carries the propagation phase exp(-j 2 pi mu_z / lam) (H(f, -mu_z) at f = 0, Eq. 4)."""
    slm = SLM(32, 40, 8e-6, 8e-6, (638e-9, 450e-9))
    sc = _phase_match_scene()
    matched = O.spectrum(sc, slm, phase_match=True)
    plain = O.spectrum(sc, slm, phase_match=False)
    r, c = slm.H // 2, slm.W // 2
    for l, lam in enumerate(slm.wavelengths):
        want = 0.0
        want_plain = 0.0 + 0.0j
        for i in range(sc.n):
            r3z = rotmat(sc.quat[i])[2, 2]
            v = sc.amp[i, l] * sc.opacity[i] * 2 * math.pi * sc.scale[i, 0] * sc.scale[i, 1] * abs(r3z)
            want += v
            want_plain += v * np.exp(-2j * math.pi * sc.mean[i, 2] / lam)
        got = matched[l, r, c]
        assert abs(got.imag) < 1e-12 * want and got.real > 0
        assert abs(got.real - want) < 1e-12 * want
        # the oracle reduces the ~6e3-cycle phase mod 1 in FP64 first: 1e-10 covers the direct exp here
        assert abs(plain[l, r, c] - want_plain) < 1e-10 * want
        # each Gaussian alone (three depths): real and positive at DC
        for i in range(sc.n):
            one = O.spectrum(sc.subset([i]), slm, phase_match=True)[l, r, c]
            assert one.real > 0 and abs(one.imag) < 1e-12 * one.real


def test_phase_match_removes_the_carrier_from_the_propagation():
    """A Gaussian moved by dz along the axis: its matched spectrum changes by the carrier-free
    propagator exp(-j 2 pi (f_z - 1/lam) dz) (the matched field keeps the reference wave's phase
    fixed at the Gaussian), while the plain spectrum changes by H(f, -dz) = exp(-j 2 pi f_z dz);
    and matched / plain = exp(+j 2 pi mu_z / lam) Gaussian by Gaussian."""
    slm = SLM(24, 30, 8e-6, 8e-6, (520e-9,))
    lam = slm.wavelengths[0]
    FX, FY, FZ = grid_freqs(slm, lam)
    sc = _phase_match_scene()
    for i in range(sc.n):
        one = sc.subset([i])
        moved = sc.subset([i])
        dz = 0.37e-3 + 0.11e-3 * i
        moved.mean[0, 2] += dz
        m0 = O.spectrum(one, slm, phase_match=True)[0]
        m1 = O.spectrum(moved, slm, phase_match=True)[0]
        p0 = O.spectrum(one, slm)[0]
        p1 = O.spectrum(moved, slm)[0]
        scale = np.abs(m0).max()
        assert np.abs(m1 - m0 * np.exp(-2j * math.pi * (FZ - 1 / lam) * dz)).max() < 1e-9 * scale
        assert np.abs(p1 - p0 * np.exp(-2j * math.pi * FZ * dz)).max() < 1e-9 * scale
        assert np.abs(m0 - p0 * np.exp(2j * math.pi * one.mean[0, 2] / lam)).max() < 1e-10 * scale


def test_phase_match_gradients_match_central_differences():
    """The backward with phase matching (its extra dL/dmu_z term) against central differences."""
    slm = SLM(20, 24, 8e-6, 8e-6, (638e-9, 450e-9))
    u = uniform_scene(17, 3, slm, scale_median_px=2.0)
    sc = make_scene(u.mean, u.quat, u.scale, u.opacity, u.amp)
    G = random_field(5, (slm.n_lambda, slm.H, slm.W)) * 1e8
    g = O.backward_spectrum(sc, slm, G, phase_match=True)

    def loss(s):
        return float(np.real(np.vdot(G, O.spectrum(s, slm, phase_match=True))))

    for field, scale in (("mean", 1e-5), ("quat", 1.0), ("opacity", 1.0)):
        arr = getattr(sc, field)
        fd = np.zeros_like(arr)
        for idx in np.ndindex(arr.shape):
            # matched, the axial phase is 2 pi (f_z - 1/lam) mu_z (|.| < 2e3 /m here) and the lateral
            # one 2 pi f_xy.mu_xy (|f_xy| < 6.3e4 /m): a 1e-10 m step keeps the truncation error < 3e-9
            h = 1e-10 if field == "mean" else 1e-6 * (abs(arr[idx]) + scale)
            sp, sm = sc.subset(np.arange(sc.n)), sc.subset(np.arange(sc.n))
            getattr(sp, field)[idx] += h
            getattr(sm, field)[idx] -= h
            fd[idx] = (loss(sp) - loss(sm)) / (2 * h)
        assert rel_l2(g[field], fd) < 1e-6, field


def test_single_terms_exponent_is_minus_log_of_the_gaussian_factor():
    """The exponent E the oracle reports per pixel (the footprint tests bound exp(-E) by the
    truncation threshold) equals -ln of the same call's |term| with the amplitude factors of Eq. 10
    divided out: |term| = 2 pi s_u s_v |r3.f| / f_z exp(-E)."""
    slm = SLM(40, 48, 8e-6, 8e-6, (520e-9,))
    lam = slm.wavelengths[0]
    FX, FY, FZ = grid_freqs(slm, lam)
    for q, s in ((qaxis([1, 0.2, 0], 0.6), (9e-6, 5e-6)), (qaxis([0, 0, 1], 0.3), (6e-6, 7e-6)),
                 (qaxis([0.3, 1, 0.1], 1.1), (4e-6, 8e-6))):
        mu = np.array([12e-6, -20e-6, 2.5e-3])
        term, E = O.single_terms(mu, q, np.array(s), lam, slm.H, slm.W, slm.pitch_x, slm.pitch_y)
        r3 = rotmat(q)[:, 2]
        g = np.abs(r3[0] * FX + r3[1] * FY + r3[2] * FZ)
        pref = 2 * math.pi * s[0] * s[1] * g / FZ
        ok = (np.abs(term) > 1e-250) & (g > 1e-6 * FZ)
        assert ok.sum() > 0.9 * ok.size
        assert np.abs(E[ok] + np.log(np.abs(term[ok]) / pref[ok])).max() < 1e-9 * max(1.0, E[ok].max())
        assert E.min() >= 0
