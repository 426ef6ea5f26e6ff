"""GPU parity of the backward splat (gws_backward, MIXED) against the FP64 oracle's gradients.

Bar: rel-L2 <= 2e-4 per parameter group (mean, quat, scale, opacity, amp), per the mixed
path's tolerance; also central differences of the GPU FP64 forward, an autograd loss through
angular-spectrum refocusing, sampled Gaussians at full size, and bitwise determinism.
"""
import math

import numpy as np
import pytest
import torch

import oracle as O
from paper_2505_06582_gb300 import gws
from paper_2505_06582_gb300.scenes import SLM, config_scene, cotangent, random_field, surface_scene, uniform_scene
from tests.helpers import grid_freqs, make_scene, rel_l2

pytestmark = pytest.mark.gpu

TOL = 2e-4
GROUPS = ("mean", "quat", "scale", "opacity", "amp")


def dev(sc):
    return gws.Gaussians.from_scene(sc, "cuda")


def _cmp(got, ref, tol=TOL):
    errs = {k: rel_l2(got[k].cpu().numpy().astype(np.float64), ref[k]) for k in GROUPS}
    for k, e in errs.items():
        assert e < tol, (k, e, errs)
    return errs


CASES = [
    ("c0", SLM(128, 128, 8e-6, 8e-6, (520e-9,)), "uniform", 0, 64),
    ("rgb_ragged", SLM(72, 100, 8e-6, 6e-6, (638e-9, 520e-9, 450e-9)), "surface", 1, 50),
    ("odd", SLM(37, 45, 8e-6, 8e-6, (520e-9,)), "uniform", 2, 12),
    ("single", SLM(40, 48, 8e-6, 8e-6, (638e-9, 450e-9)), "uniform", 3, 1),
    # 97 rows = two 48-row tiles and a last tile of one row
    ("one_row_tail", SLM(97, 70, 8e-6, 6e-6, (520e-9,)), "surface", 4, 40),
]


@pytest.mark.parametrize("name,slm,kind,seed,n", CASES, ids=[c[0] for c in CASES])
@pytest.mark.parametrize("domain", [gws.DOMAIN_FIELD, gws.DOMAIN_SPECTRUM], ids=["field", "spectrum"])
def test_backward_matches_oracle(name, slm, kind, seed, n, domain):
    sc = uniform_scene(seed, n, slm) if kind == "uniform" else surface_scene(seed, n, slm, n_surfaces=3)
    G = cotangent(100 + seed, slm)  # complex64, the same values go to both sides
    got = gws.backward(dev(sc), slm, torch.as_tensor(G, device="cuda"), domain=domain)
    if domain == gws.DOMAIN_FIELD:
        ref = O.backward_field(sc, slm, G.astype(np.complex128))
    else:
        ref = O.backward_spectrum(sc, slm, G.astype(np.complex128))
    _cmp(got, ref)


def test_backward_phase_match():
    slm = SLM(48, 64, 8e-6, 8e-6, (520e-9, 450e-9))
    sc = uniform_scene(5, 16, slm)
    G = cotangent(7, slm)
    got = gws.backward(dev(sc), slm, torch.as_tensor(G, device="cuda"), domain=gws.DOMAIN_SPECTRUM, phase_match=True)
    ref = O.backward_spectrum(sc, slm, G.astype(np.complex128), phase_match=True)
    _cmp(got, ref)


def test_backward_where_g_changes_sign_inside_tiles():
    """Nearly edge-on Gaussians (|r3_z| <= 0.02): the zero line of g = r3.f crosses the grid, so some
    (Gaussian, 64 x 64 tile) pairs see both signs of g and take the per-pixel sign, the rest keep one sign
    (positive and negative) and take it once per tile; the gradients must match the oracle's."""
    from paper_2505_06582_gb300.scenes import _quat_from_frame, _tangent_frame
    slm = SLM(128, 160, 8e-6, 8e-6, (520e-9, 638e-9))
    rng = np.random.default_rng(41)
    n = 12
    r3z = np.array([0.002, -0.002, 0.006, -0.006, 0.01, -0.01, 0.014, -0.014, 0.018, -0.018, 0.02, -0.02])
    psi = rng.uniform(0, 2 * np.pi, n)  # direction of the in-plane part of the normal
    rxy = np.sqrt(1 - r3z ** 2)
    normal = np.stack([rxy * np.cos(psi), rxy * np.sin(psi), r3z], 1)
    r1, r2, r3 = _tangent_frame(normal, rng.uniform(0, np.pi, n))
    quat = _quat_from_frame(r1, r2, r3).astype(np.float32)
    ax, ay = slm.W * slm.pitch_x, slm.H * slm.pitch_y
    mean = np.stack([rng.uniform(-ax / 3, ax / 3, n), rng.uniform(-ay / 3, ay / 3, n), rng.uniform(1e-3, 4e-3, n)], 1)
    sc = make_scene(mean, quat, rng.uniform(2, 5, (n, 2)) * 8e-6, rng.uniform(0.3, 1.0, n),
                    rng.uniform(0.2, 1.0, (n, 2)))
    sc.quat = sc.quat.astype(np.float32)
    sc.scale, sc.opacity, sc.amp = sc.scale.astype(np.float32), sc.opacity.astype(np.float32), sc.amp.astype(np.float32)
    # the scene does what it is for: per wavelength, tiles where g keeps each sign and tiles where it changes
    q = sc.quat.astype(np.float64) / np.linalg.norm(sc.quat.astype(np.float64), axis=1, keepdims=True)
    w, x, y, z = q.T
    n3 = np.stack([2 * (x * z + w * y), 2 * (y * z - w * x), 1 - 2 * (x * x + y * y)], 1)
    kinds = set()
    for lam in slm.wavelengths:
        FX, FY, FZ = grid_freqs(slm, lam)
        for i in range(n):
            gi = n3[i, 0] * FX + n3[i, 1] * FY + n3[i, 2] * FZ
            for r0 in range(0, slm.H, 64):
                for c0 in range(0, slm.W, 64):
                    t = gi[r0:r0 + 64, c0:c0 + 64]
                    kinds.add("mixed" if t.min() < 0 < t.max() else ("pos" if t.min() > 0 else "neg"))
    assert kinds == {"mixed", "pos", "neg"}, kinds
    G = cotangent(43, slm)
    got = gws.backward(dev(sc), slm, torch.as_tensor(G, device="cuda"))
    _cmp(got, O.backward_field(sc, slm, G.astype(np.complex128)))
    u = gws.forward(dev(sc), slm, domain=gws.DOMAIN_SPECTRUM).cpu().numpy()
    assert rel_l2(u, O.spectrum(sc, slm)) < TOL


def test_backward_is_deterministic():
    slm = SLM(96, 128, 8e-6, 8e-6, (638e-9, 520e-9))
    sc = surface_scene(8, 400, slm, n_surfaces=4)
    G = torch.as_tensor(cotangent(9, slm), device="cuda")
    a = gws.backward(dev(sc), slm, G)
    b = gws.backward(dev(sc), slm, G)
    for k in GROUPS:
        assert torch.equal(a[k], b[k]), k


def test_backward_empty_and_unsupported():  # FP64 backward is not provided
    slm = SLM(16, 16, 8e-6, 8e-6, (520e-9,))
    sc = uniform_scene(10, 3, slm)
    G = torch.as_tensor(cotangent(1, slm), device="cuda")
    e = sc.subset(np.arange(0))
    out = gws.backward(dev(e), slm, G)
    assert out["mean"].numel() == 0
    with pytest.raises(gws.GwsError) as ei:
        gws.backward(dev(sc), slm, G, prec=gws.PREC_FP64)
    assert ei.value.code == 6


def test_backward_matches_central_differences_of_the_fp64_forward():
    """L(theta) = Re<G, u_SLM(theta)> evaluated with the GPU FP64 path; central differences
    on every parameter of a 3-Gaussian scene against the MIXED backward."""
    slm = SLM(24, 32, 8e-6, 8e-6, (638e-9, 450e-9))
    u = uniform_scene(11, 3, slm, scale_median_px=2.0)
    sc = make_scene(u.mean, u.quat, u.scale, u.opacity, u.amp)
    G = random_field(12, (2, 24, 32)).astype(np.complex64)
    Gt = torch.as_tensor(G.astype(np.complex128), device="cuda")

    def loss(s):
        g = gws.Gaussians(torch.tensor(s.mean, dtype=torch.float64, device="cuda"),
                          torch.tensor(s.quat, dtype=torch.float32, device="cuda"),
                          torch.tensor(s.scale, dtype=torch.float32, device="cuda"),
                          torch.tensor(s.opacity, dtype=torch.float32, device="cuda"),
                          torch.tensor(s.amp, dtype=torch.float32, device="cuda"))
        U = gws.forward(g, slm, prec=gws.PREC_FP64, domain=gws.DOMAIN_SPECTRUM)
        return float((Gt.conj() * U).real.sum())

    got = gws.backward(dev(sc), slm, torch.as_tensor(G, device="cuda"), domain=gws.DOMAIN_SPECTRUM)
    # float32 parameters: perturb by steps representable in float32 and difference in FP64
    for field in GROUPS:
        arr = getattr(sc, field)
        fd = np.zeros_like(arr)
        for idx in np.ndindex(arr.shape):
            base = arr[idx]
            h = 1e-11 if field == "mean" else 2e-3 * (abs(base) + (1e-5 if field == "scale" else 0.1))
            sp = sc.subset(np.arange(sc.n))
            sm = sc.subset(np.arange(sc.n))
            getattr(sp, field)[idx] = np.float32(base + h) if field != "mean" else base + h
            getattr(sm, field)[idx] = np.float32(base - h) if field != "mean" else base - h
            hp = getattr(sp, field)[idx] - base
            hm = base - getattr(sm, field)[idx]
            fd[idx] = (loss(sp) - loss(sm)) / (hp + hm)
        e = rel_l2(got[field].cpu().numpy().astype(np.float64), fd)
        assert e < 5e-4, (field, e)


def _refocus_intensity_loss(u, slm, targets, zs):
    """sum_z sum_l || |ASM(u, +z)|^2 - t ||^2 (angular-spectrum refocus of the SLM field)."""
    tot = 0
    for l, lam in enumerate(slm.wavelengths):
        FX, FY, FZ = (torch.as_tensor(a, device=u.device) for a in grid_freqs(slm, lam))
        U = torch.fft.fftshift(torch.fft.fft2(torch.fft.ifftshift(u[l])))
        for k, z in enumerate(zs):
            Hz = torch.exp(2j * math.pi * z * FZ.to(torch.float64)).to(U.dtype)
            uz = torch.fft.fftshift(torch.fft.ifft2(torch.fft.ifftshift(U * Hz)))
            tot = tot + ((uz.abs() ** 2 - targets[l][k]) ** 2).sum()
    return tot


def test_autograd_refocus_loss_matches_oracle():
    """The differentiable workload's loss (refocus at z = 2, 5, 8 mm, seeded targets) at a
    small size: autograd through GWSFunction vs the oracle's gradients for the same loss,
    whose field cotangent is computed from the oracle's own field."""
    slm = SLM(64, 80, 8e-6, 8e-6, (638e-9, 520e-9, 450e-9))
    sc = surface_scene(4, 60, slm, n_surfaces=3)
    zs = (2e-3, 5e-3, 8e-3)
    rng = np.random.default_rng(4)
    uref = O.field(sc, slm)
    targets = [[rng.uniform(0, 1, (slm.H, slm.W)) * np.mean(np.abs(uref[l]) ** 2) for _ in zs] for l in range(3)]
    # oracle: dL/du from the oracle's field (CPU, FP64), then the oracle's backward
    ut = torch.tensor(uref, requires_grad=True)
    Lref = _refocus_intensity_loss(ut, slm, [[torch.tensor(t) for t in tl] for tl in targets], zs)
    Lref.backward()
    ref = O.backward_field(sc, slm, ut.grad.numpy())
    # GPU: autograd through the library
    p = {k: torch.tensor(getattr(sc, k), dtype=torch.float64 if k == "mean" else torch.float32, device="cuda",
                         requires_grad=True) for k in GROUPS}
    u = gws.gws_field(p["mean"], p["quat"], p["scale"], p["opacity"], p["amp"], slm)
    L = _refocus_intensity_loss(u.to(torch.complex128), slm,
                                [[torch.tensor(t, device="cuda") for t in tl] for tl in targets], zs)
    L.backward()
    assert abs(L.item() - Lref.item()) < 1e-4 * abs(Lref.item())
    _cmp({k: p[k].grad for k in GROUPS}, ref)


def _spread_over_footprint_radius(sc, k, seed):
    """k Gaussians spread over the spectral footprint's largest radius (1 / the smallest singular value
    of the projected factor M = [s_u r1_xy, s_v r2_xy], Eq. 10's Gaussian factor at the reference
    frequency), always including the widest and the narrowest footprint."""
    q = sc.quat / np.linalg.norm(sc.quat, axis=1, keepdims=True)
    w, x, y, z = q.T
    r1 = np.stack([1 - 2 * (y * y + z * z), 2 * (x * y + w * z)], 1)
    r2 = np.stack([2 * (x * y - w * z), 1 - 2 * (x * x + z * z)], 1)
    M = np.stack([sc.scale[:, :1] * r1, sc.scale[:, 1:] * r2], 2)  # [n][xy][uv]
    smin = np.linalg.svd(M, compute_uv=False)[:, -1]
    R = 1.0 / np.maximum(smin, 1e-30)
    order = np.argsort(R)
    qs = np.linspace(0, len(order) - 1, k - 2).round().astype(int)
    rng = np.random.default_rng(seed)
    pick = set(order[qs].tolist()) | {int(order[0]), int(order[-1])}
    while len(pick) < k:
        pick.add(int(rng.integers(0, sc.n)))
    return np.array(sorted(pick)), R


@pytest.mark.parametrize("cfg", ["c4_differentiable", "headline_1m_1080p_3l", "c2_precision_at_scale"])
def test_full_size_backward_sampled_gaussians(cfg):
    """Gradients of 36 Gaussians of a full-size scene (spread over footprint radius, the widest and the
    narrowest included) against the oracle's gradients of the same Gaussians, per parameter group."""
    sc, slm = config_scene(cfg)
    G = cotangent(21, slm)
    got = gws.backward(dev(sc), slm, torch.as_tensor(G, device="cuda"), domain=gws.DOMAIN_SPECTRUM)
    which, R = _spread_over_footprint_radius(sc, 36, 3)
    ref = O.backward_spectrum_at(sc, slm, G.astype(np.complex128), which)
    for k in GROUPS:
        e = rel_l2(got[k].cpu().numpy()[which].astype(np.float64), ref[k])
        assert e < TOL, (k, e)
    # the extremes on their own (the widest footprint spans the grid, the narrowest a few tiles): no
    # outlier, i.e. each one's error within the group's tolerance times the group's RMS over the sample
    # (a single Gaussian's gradient can itself be a near-cancelling sum, e.g. dL/do of an edge-on one)
    for i in (int(np.argmax(R[which])), int(np.argmin(R[which]))):
        for k in GROUPS:
            err = np.linalg.norm(got[k].cpu().numpy()[which[i]].astype(np.float64) - ref[k][i])
            rms = np.linalg.norm(ref[k]) / np.sqrt(len(which))
            assert err < TOL * rms, (k, "extreme", R[which[i]], err / rms)


# ---------------------------------------------------------------------------------------
# depth-sorted transmittance: cross terms through T_i
# ---------------------------------------------------------------------------------------

def test_backward_sorted_t_matches_oracle():
    slm = SLM(64, 72, 8e-6, 8e-6, (638e-9, 520e-9))
    sc = surface_scene(50, 60, slm, n_surfaces=2, scale_median_px=5.0)
    T = O.transmittance(sc)
    assert (T < 0.95).sum() > 10  # the cross terms matter
    G = cotangent(51, slm)
    got = gws.backward(dev(sc), slm, torch.as_tensor(G, device="cuda"), blend=gws.BLEND_SORTED_T)
    ref = O.backward_field(sc, slm, G.astype(np.complex128), blend=O.BLEND_SORTED_T)
    _cmp(got, ref)
    # and the cross terms are not negligible: the order-invariant gradients differ
    oit = O.backward_field(sc, slm, G.astype(np.complex128), blend=O.BLEND_OIT)
    assert rel_l2(oit["mean"], ref["mean"]) > 1e-2


def test_backward_sorted_t_matches_central_differences():
    from tests.helpers import qaxis
    slm = SLM(20, 24, 8e-6, 8e-6, (638e-9, 450e-9))
    sc = make_scene([[0, 0, 2e-3], [12e-6, -6e-6, 3e-3], [-8e-6, 10e-6, 4e-3]],
                    [qaxis([1, 0.4, 0], 0.5), qaxis([0.3, 1, 0], 0.4), qaxis([0, 0, 1], 1.0)],
                    [[25e-6, 18e-6], [20e-6, 22e-6], [15e-6, 17e-6]], [0.8, 0.6, 0.7],
                    [[0.9, 0.4], [0.5, 0.8], [0.7, 0.6]])
    G = random_field(52, (2, 20, 24)).astype(np.complex64)
    Gt = torch.as_tensor(G.astype(np.complex128), device="cuda")

    def loss(s):
        g = gws.Gaussians(torch.tensor(s.mean, dtype=torch.float64, device="cuda"),
                          torch.tensor(s.quat, dtype=torch.float32, device="cuda"),
                          torch.tensor(s.scale, dtype=torch.float32, device="cuda"),
                          torch.tensor(s.opacity, dtype=torch.float32, device="cuda"),
                          torch.tensor(s.amp, dtype=torch.float32, device="cuda"))
        U = gws.forward(g, slm, prec=gws.PREC_FP64, domain=gws.DOMAIN_SPECTRUM, blend=gws.BLEND_SORTED_T)
        return float((Gt.conj() * U).real.sum())

    got = gws.backward(dev(sc), slm, torch.as_tensor(G, device="cuda"), domain=gws.DOMAIN_SPECTRUM,
                       blend=gws.BLEND_SORTED_T)
    for field in GROUPS:
        arr = getattr(sc, field)
        fd = np.zeros_like(arr)
        for idx in np.ndindex(arr.shape):
            base = arr[idx]
            h = 1e-11 if field == "mean" else 2e-3 * (abs(base) + (1e-5 if field == "scale" else 0.1))
            sp = sc.subset(np.arange(sc.n))
            sm = sc.subset(np.arange(sc.n))
            getattr(sp, field)[idx] = np.float32(base + h) if field != "mean" else base + h
            getattr(sm, field)[idx] = np.float32(base - h) if field != "mean" else base - h
            fd[idx] = (loss(sp) - loss(sm)) / ((getattr(sp, field)[idx] - base) + (base - getattr(sm, field)[idx]))
        e = rel_l2(got[field].cpu().numpy().astype(np.float64), fd)
        assert e < 5e-4, (field, e)
