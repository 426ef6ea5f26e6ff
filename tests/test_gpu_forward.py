"""GPU parity: the CUDA forward path (through the C ABI) against the FP64 oracle.

Bars (relative L2 over each wavelength's field or spectrum):
  FP64 GPU path <= 1e-6, mixed-precision path <= 2e-4.
Depth order: bit-exact.  Transmittance: FP64 both sides (the 1/255 decisions are taken
in FP64 on both sides), 1e-12.
"""
import math

import numpy as np
import pytest
import torch

import oracle as O
from paper_2505_06582_gb300 import gws
from paper_2505_06582_gb300.scenes import SLM, config_scene, surface_scene, uniform_scene
from tests.helpers import make_scene, qaxis, rel_l2

pytestmark = pytest.mark.gpu

TOL64, TOLMX = 1e-6, 2e-4


def per_lambda_rel(a, b):
    return [rel_l2(a[l], b[l]) for l in range(b.shape[0])]


def dev(sc):
    return gws.Gaussians.from_scene(sc, "cuda")


# ---------------------------------------------------------------------------------------
# element-wise parity at oracle-sized workloads (several tiles, ragged tails)
# ---------------------------------------------------------------------------------------

CASES = [
    ("c0", SLM(128, 128, 8e-6, 8e-6, (520e-9,)), "uniform", 0, 64),
    ("ragged", SLM(100, 150, 8e-6, 6e-6, (638e-9, 450e-9)), "uniform", 3, 40),
    ("odd", SLM(77, 99, 8e-6, 8e-6, (520e-9,)), "surface", 4, 60),
    ("tiny", SLM(9, 7, 8e-6, 8e-6, (520e-9,)), "uniform", 5, 3),
    ("onecol", SLM(33, 1, 8e-6, 8e-6, (520e-9,)), "uniform", 6, 4),
]


def _scene(kind, seed, n, slm):
    if kind == "uniform":
        return uniform_scene(seed, n, slm)
    return surface_scene(seed, n, slm, n_surfaces=4)


@pytest.mark.parametrize("name,slm,kind,seed,n", CASES, ids=[c[0] for c in CASES])
@pytest.mark.parametrize("blend", [gws.BLEND_OIT, gws.BLEND_SORTED_T], ids=["oit", "sortedT"])
def test_forward_field_matches_oracle(name, slm, kind, seed, n, blend):
    sc = _scene(kind, seed, n, slm)
    ref = O.field(sc, slm, blend=blend)
    g = dev(sc)
    f64 = gws.forward(g, slm, prec=gws.PREC_FP64, blend=blend).cpu().numpy()
    fmx = gws.forward(g, slm, prec=gws.PREC_MIXED, blend=blend).cpu().numpy()
    assert max(per_lambda_rel(f64, ref)) < TOL64
    assert max(per_lambda_rel(fmx, ref)) < TOLMX


@pytest.mark.parametrize("tile_cfg", list(range(1, 13)))
def test_spectrum_domain_and_every_tile_config(tile_cfg):
    slm = SLM(96, 160, 8e-6, 8e-6, (638e-9, 520e-9, 450e-9))
    sc = surface_scene(7, 120, slm, n_surfaces=3)
    ref = O.spectrum(sc, slm)
    g = dev(sc)
    u = gws.forward(g, slm, prec=gws.PREC_MIXED, domain=gws.DOMAIN_SPECTRUM, tile_cfg=tile_cfg).cpu().numpy()
    assert max(per_lambda_rel(u, ref)) < TOLMX
    u64 = gws.forward(g, slm, prec=gws.PREC_FP64, domain=gws.DOMAIN_SPECTRUM).cpu().numpy()
    assert max(per_lambda_rel(u64, ref)) < TOL64


def _near_slm(sc, lo, hi, seed):
    """The scene with its depths redrawn in [lo, hi] (m)."""
    sc.mean[:, 2] = np.random.default_rng(seed).uniform(lo, hi, sc.n)
    return sc


# grids where the column step's residual |t_z dl| stays below its 2e-3 rad bound for depths
# up to 0.15 mm (ragged widths, an odd grid, a pitch with evanescent corners), and the phase match
STEP_CASES = [
    ("96x160", SLM(96, 160, 8e-6, 8e-6, (638e-9, 520e-9, 450e-9)), 0.15e-3, False),
    ("ragged", SLM(100, 150, 8e-6, 6e-6, (638e-9, 450e-9)), 0.1e-3, False),
    ("odd", SLM(77, 99, 8e-6, 8e-6, (520e-9,)), 0.15e-3, True),
    ("evanescent", SLM(64, 72, 0.3e-6, 0.3e-6, (520e-9,)), 0.4e-6, False),
]


@pytest.mark.parametrize("name,slm,zmax,pm", STEP_CASES, ids=[c[0] for c in STEP_CASES])
@pytest.mark.parametrize("tile_cfg", [11, 12])
def test_column_step_configs_match_oracle(name, slm, zmax, pm, tile_cfg):
    """The column-step configurations on grids where their step path runs (the records' residual
    phase steps within bounds; at the evanescent boundary, where f_z bends sharply, those tiles
    take the direct path): element-wise against the oracle, bar 2e-4 per wavelength."""
    if name == "evanescent":
        sc = uniform_scene(12, 30, slm)
        sc.scale[:] = np.float32(0.6e-6)
    else:
        sc = surface_scene(11, 150, slm, n_surfaces=3)
    sc = _near_slm(sc, 0.2 * zmax, zmax, 13)
    ref = O.spectrum(sc, slm, phase_match=pm)
    u = gws.forward(dev(sc), slm, prec=gws.PREC_MIXED, domain=gws.DOMAIN_SPECTRUM, tile_cfg=tile_cfg,
                    phase_match=pm).cpu().numpy()
    assert max(per_lambda_rel(u, ref)) < TOLMX, per_lambda_rel(u, ref)


def test_column_step_mixed_chunks_at_512x768():
    """A 512 x 768 grid with 1200 Gaussians at 2-10 mm: some records' residual phase step is
    within the column step's bound and some not, so chunks of both kinds run in one launch.
    Sampled spectrum against the oracle (2e-4 per wavelength) and the whole spectrum against the
    direct configuration of the same tile shape."""
    slm = SLM(512, 768, 8e-6, 8e-6, (638e-9, 520e-9, 450e-9))
    sc = surface_scene(14, 1200, slm, n_surfaces=6)
    g = dev(sc)
    lam, r, c = _samples(slm, 1500, 15)
    ref = O.spectrum_at(sc, slm, lam, r, c)
    u1 = gws.forward(g, slm, prec=gws.PREC_MIXED, domain=gws.DOMAIN_SPECTRUM, tile_cfg=1)
    for cfg in (11, 12):
        u = gws.forward(g, slm, prec=gws.PREC_MIXED, domain=gws.DOMAIN_SPECTRUM, tile_cfg=cfg)
        got = u[torch.as_tensor(lam, dtype=torch.long), torch.as_tensor(r, dtype=torch.long),
                torch.as_tensor(c, dtype=torch.long)].cpu().numpy()
        for l in range(slm.n_lambda):
            m = lam == l
            assert rel_l2(got[m], ref[m]) < TOLMX, (cfg, l, rel_l2(got[m], ref[m]))
        for l in range(slm.n_lambda):
            e = (torch.linalg.norm(u[l] - u1[l]) / torch.linalg.norm(u1[l])).item()
            assert e < 2e-5, (cfg, l, e)


def test_phase_match_option():
    slm = SLM(64, 64, 8e-6, 8e-6, (520e-9,))
    sc = uniform_scene(8, 20, slm)
    ref = O.spectrum(sc, slm, phase_match=True)
    g = dev(sc)
    for prec, tol in ((gws.PREC_FP64, TOL64), (gws.PREC_MIXED, TOLMX)):
        u = gws.forward(g, slm, prec=prec, domain=gws.DOMAIN_SPECTRUM, phase_match=True).cpu().numpy()
        assert rel_l2(u, ref) < tol


def test_empty_and_single_gaussian():
    slm = SLM(40, 56, 8e-6, 8e-6, (520e-9, 450e-9))
    sc = uniform_scene(9, 1, slm)
    empty = sc.subset(np.arange(0))
    for prec in (gws.PREC_FP64, gws.PREC_MIXED):
        z = gws.forward(dev(empty), slm, prec=prec).cpu().numpy()
        assert np.array_equal(z, np.zeros_like(z))
        u = gws.forward(dev(sc), slm, prec=prec).cpu().numpy()
        assert max(per_lambda_rel(u, O.field(sc, slm))) < (TOL64 if prec == gws.PREC_FP64 else TOLMX)


def test_evanescent_band_is_zero():
    # pitch below lambda/2: the corners of the grid are evanescent (Eq. 4 cuts them)
    slm = SLM(32, 32, 0.2e-6, 0.2e-6, (520e-9,))
    sc = make_scene([[0, 0, 2e-6]], [qaxis([1, 0, 0], 0.4)], [[0.3e-6, 0.4e-6]], [1.0], [[1.0]])
    ref = O.spectrum(sc, slm)
    assert (ref == 0).any() and (ref != 0).any()
    for prec, tol in ((gws.PREC_FP64, TOL64), (gws.PREC_MIXED, TOLMX)):
        u = gws.forward(dev(sc), slm, prec=prec, domain=gws.DOMAIN_SPECTRUM).cpu().numpy()
        assert rel_l2(u, ref) < tol
        assert np.all(u[ref == 0] == 0)


def test_full_occlusion_sorted_t():
    slm = SLM(64, 64, 8e-6, 8e-6, (520e-9,))
    front = make_scene([[0, 0, 2e-3]], [[1, 0, 0, 0]], [[80e-6, 60e-6]], [1.0], [[0.7]])
    rear = make_scene([[0, 0, 4e-3]], [qaxis([1, 0, 0], 0.5)], [[20e-6, 20e-6]], [0.8], [[0.9]])
    both = rear.concat(front)
    for prec in (gws.PREC_FP64, gws.PREC_MIXED):
        u = gws.forward(dev(both), slm, prec=prec, blend=gws.BLEND_SORTED_T, domain=gws.DOMAIN_SPECTRUM)
        uf = gws.forward(dev(front), slm, prec=prec, domain=gws.DOMAIN_SPECTRUM)
        assert torch.equal(u, uf)


# ---------------------------------------------------------------------------------------
# depth sort, transmittance, footprints
# ---------------------------------------------------------------------------------------

def test_depth_order_bit_exact_with_ties():
    slm = SLM(8, 8, 8e-6, 8e-6, (520e-9,))
    sc = uniform_scene(10, 5000, slm)
    sc.mean[::7, 2] = 3e-3
    sc.mean[3, 2] = -0.0
    sc.mean[4, 2] = 0.0
    sc.mean[5, 2] = -1e-3
    order = gws.depth_order(dev(sc)).cpu().numpy()
    assert np.array_equal(order, O.depth_order(sc.mean))


def test_transmittance_matches_oracle():
    slm = SLM(64, 64, 8e-6, 8e-6, (520e-9,))
    sc = surface_scene(11, 3000, slm, n_surfaces=3, scale_median_px=6.0)
    T = gws.transmittance(dev(sc)).cpu().numpy()
    Tr = O.transmittance(sc)
    assert (Tr < 0.99).mean() > 0.2  # the scene really occludes
    assert np.abs(T - Tr).max() < 1e-12


def test_footprints_bound_the_truncated_spectrum():
    """Outside each footprint ellipse the oracle's Gaussian factor exp(-E) is below eps."""
    slm = SLM(128, 160, 8e-6, 8e-6, (638e-9, 450e-9))
    sc = surface_scene(12, 40, slm, n_surfaces=2)
    eps = 1e-5
    fx = (np.arange(slm.W) - slm.W // 2) / (slm.W * slm.pitch_x)
    fy = (np.arange(slm.H) - slm.H // 2) / (slm.H * slm.pitch_y)
    FX, FY = np.meshgrid(fx, fy)
    for l, lam in enumerate(slm.wavelengths):
        ell = gws.footprints(dev(sc), slm, l, trunc_eps=eps).cpu().numpy().astype(np.float64)
        for i in range(sc.n):
            _, E = O.single_terms(sc.mean[i], sc.quat[i], sc.scale[i], lam, slm.H, slm.W, slm.pitch_x, slm.pitch_y)
            q = ell[i, 0] * FX ** 2 + 2 * ell[i, 1] * FX * FY + ell[i, 2] * FY ** 2
            outside = q > 1.0
            assert np.all(E[outside] >= math.log(1 / eps) * (1 - 1e-6))


# ---------------------------------------------------------------------------------------
# batching, device status
# ---------------------------------------------------------------------------------------

def test_batched_equals_individual_calls_bitwise():
    slm = SLM(72, 96, 8e-6, 8e-6, (638e-9, 520e-9))
    scenes = [surface_scene(20 + k, n, slm, n_surfaces=2) for k, n in enumerate([30, 1, 75, 0, 12])]
    gs = [dev(s) for s in scenes]
    for prec in (gws.PREC_MIXED, gws.PREC_FP64):
        for blend in (gws.BLEND_OIT, gws.BLEND_SORTED_T):
            outs = gws.forward_batched(gs, slm, prec=prec, blend=blend)
            for g, o in zip(gs, outs):
                single = gws.forward(g, slm, prec=prec, blend=blend)
                assert torch.equal(o, single)


def test_device_status_reports_bad_inputs_and_timeouts():
    slm = SLM(32, 32, 8e-6, 8e-6, (520e-9,))
    sc = uniform_scene(13, 10, slm)
    ws = torch.empty(gws.workspace_size([10], gws.Slm.of(slm), gws.make_opts()) + 4096, dtype=torch.uint8,
                     device="cuda")
    gws.forward(dev(sc), slm, workspace=ws)
    assert gws.device_status([10], slm, workspace=ws) == 0
    bad = sc.subset(np.arange(10))
    bad.mean[3, 1] = np.nan
    gws.forward(dev(bad), slm, workspace=ws)
    assert gws.device_status([10], slm, workspace=ws) == 4
    bad = sc.subset(np.arange(10))
    bad.opacity[2] = 1.5
    gws.forward(dev(bad), slm, workspace=ws)
    assert gws.device_status([10], slm, workspace=ws) == 1
    # a bounded wait that nothing completes: the kernel records TIMEOUT and returns
    gws.forward(dev(sc), slm, workspace=ws, debug_flags=gws.DEBUG_FORCE_TIMEOUT, timeout_cycles=200_000)
    assert gws.device_status([10], slm, workspace=ws) == 5
    # the context is intact: a normal call afterwards is correct
    u = gws.forward(dev(sc), slm, workspace=ws).cpu().numpy()
    assert gws.device_status([10], slm, workspace=ws) == 0
    assert rel_l2(u, O.field(sc, slm)) < TOLMX


# ---------------------------------------------------------------------------------------
# full-size workloads: sampled spectra (the oracle computes each sample over all Gaussians)
# ---------------------------------------------------------------------------------------

def _samples(slm, k, seed):
    rng = np.random.default_rng(seed)
    lam = rng.integers(0, slm.n_lambda, k).astype(np.int32)
    # half near DC (where every Gaussian contributes), half anywhere
    r = np.where(np.arange(k) % 2 == 0, rng.integers(0, slm.H, k),
                 slm.H // 2 + rng.integers(-slm.H // 8, slm.H // 8, k)).astype(np.int32)
    c = np.where(np.arange(k) % 2 == 0, rng.integers(0, slm.W, k),
                 slm.W // 2 + rng.integers(-slm.W // 8, slm.W // 8, k)).astype(np.int32)
    return lam, r, c


@pytest.mark.parametrize("cfg,n,k", [("c1_slm_size", None, 400), ("headline_1m_1080p_3l", None, 120)])
def test_full_size_sampled_spectrum(cfg, n, k):
    sc, slm = config_scene(cfg, n=n)
    g = dev(sc)
    u = gws.forward(g, slm, prec=gws.PREC_MIXED, domain=gws.DOMAIN_SPECTRUM)
    lam, r, c = _samples(slm, k, 99)
    got = u[torch.as_tensor(lam, dtype=torch.long), torch.as_tensor(r, dtype=torch.long),
            torch.as_tensor(c, dtype=torch.long)].cpu().numpy()
    ref = O.spectrum_at(sc, slm, lam, r, c)
    for l in range(slm.n_lambda):
        m = lam == l
        assert rel_l2(got[m], ref[m]) < TOLMX, (l, rel_l2(got[m], ref[m]))
    # the field of the same call equals torch's FFT of the spectrum (the IDFT stage at full size)
    f = gws.forward(g, slm, prec=gws.PREC_MIXED)
    dfx, dfy = 1 / (slm.W * slm.pitch_x), 1 / (slm.H * slm.pitch_y)
    uu = u.to(torch.complex128)
    ref_f = dfx * dfy * slm.H * slm.W * torch.fft.fftshift(torch.fft.ifft2(torch.fft.ifftshift(uu, dim=(-2, -1))),
                                                           dim=(-2, -1))
    for l in range(slm.n_lambda):
        e = (torch.linalg.norm(f[l].to(torch.complex128) - ref_f[l]) / torch.linalg.norm(ref_f[l])).item()
        assert e < 1e-5, e


def _band_samples(slm, band, k, seed):
    """k frequencies of one band: 'dc' (within 2 pixels of f = 0), 'mid' (normalised radius in
    [0.3, 0.6] of the grid's half extent per axis), 'outer' ([0.8, 1.0]: where few footprints reach
    and the truncation acts) or 'corner' (corners of the forward's 64 x 32 frequency tiles, where the
    in-tile phase deltas from the tile's reference frequency are largest)."""
    rng = np.random.default_rng(seed)
    H, W = slm.H, slm.W
    if band == "dc":
        r = H // 2 + rng.integers(-2, 3, k)
        c = W // 2 + rng.integers(-2, 3, k)
    elif band == "corner":
        r = rng.integers(0, (H + 31) // 32, k) * 32 + rng.choice([0, 31], k)
        c = rng.integers(0, (W + 63) // 64, k) * 64 + rng.choice([0, 63], k)
        r, c = np.minimum(r, H - 1), np.minimum(c, W - 1)
    else:
        lo, hi = (0.3, 0.6) if band == "mid" else (0.8, 1.0)
        rad = rng.uniform(lo, hi, k)
        ang = rng.uniform(0, 2 * math.pi, k)
        r = np.clip(np.round(H // 2 + rad * np.sin(ang) * (H // 2)), 0, H - 1)
        c = np.clip(np.round(W // 2 + rad * np.cos(ang) * (W // 2)), 0, W - 1)
    return r.astype(np.int32), c.astype(np.int32)


@pytest.mark.parametrize("cfg", ["headline_1m_1080p_3l", "c2_precision_at_scale"])
def test_full_size_band_stratified_spectrum(cfg):
    """Full-size parity per frequency band and wavelength, each band against its own norm: the
    sampled mixed spectrum vs the oracle, which sums every Gaussian at each sample without
    truncation; for the direct configuration 1 and the column-step configuration 11 (the
    autotuner's candidates for the bench's launch)."""
    sc, slm = config_scene(cfg)
    g = dev(sc)
    us = {t: gws.forward(g, slm, prec=gws.PREC_MIXED, domain=gws.DOMAIN_SPECTRUM, tile_cfg=t) for t in (1, 11)}
    report = {}
    for bi, band in enumerate(("dc", "mid", "outer", "corner")):
        for l in range(slm.n_lambda):
            r, c = _band_samples(slm, band, 40, 1000 + 10 * bi + l)
            lam = np.full(r.shape, l, np.int32)
            ref = O.spectrum_at(sc, slm, lam, r, c)
            peak = np.abs(ref).max()
            for t, u in us.items():
                got = u[l, torch.as_tensor(r, dtype=torch.long), torch.as_tensor(c, dtype=torch.long)].cpu().numpy()
                e = rel_l2(got, ref)
                report[(t, band, l)] = (e, float(np.abs(got - ref).max() / peak), float(peak))
                assert e < TOLMX, (t, band, l, e)
    print(cfg, {f"cfg{t}/{b}/{l}": f"rel-L2 {v[0]:.2e}, max|err|/peak {v[1]:.2e}, peak {v[2]:.3g}"
                for (t, b, l), v in report.items()})


def test_fp64_path_at_slm_size_sampled():
    sc, slm = config_scene("c1_slm_size", n=2000)
    u = gws.forward(dev(sc), slm, prec=gws.PREC_FP64, domain=gws.DOMAIN_SPECTRUM)
    lam, r, c = _samples(slm, 300, 5)
    got = u[torch.as_tensor(lam, dtype=torch.long), torch.as_tensor(r, dtype=torch.long),
            torch.as_tensor(c, dtype=torch.long)].cpu().numpy()
    ref = O.spectrum_at(sc, slm, lam, r, c)
    assert rel_l2(got, ref) < TOL64


# ---------------------------------------------------------------------------------------
# encoding
# ---------------------------------------------------------------------------------------

def _circ(a, b):
    return np.abs(np.angle(np.exp(1j * (a - b))))


@pytest.mark.parametrize("shape", [(1, 64, 64), (3, 37, 53), (2, 1080, 1920)])
def test_encode_matches_oracle(shape):
    from paper_2505_06582_gb300.scenes import random_field
    f = random_field(17, shape, zero_frac=0.01)
    slm = SLM(shape[1], shape[2], 8e-6, 8e-6, tuple([520e-9] * shape[0]))
    # FP64 field: FP64 encode, written as float32 phases: half an ulp of |P| <= pi is 1.2e-7 rad
    p64 = gws.encode(torch.as_tensor(f, device="cuda"), slm).cpu().numpy()
    ref = O.encode(f)
    assert _circ(p64, ref).max() < 2.5e-7
    # complex64 field: FP32 encode.  acos is ill-conditioned near a = 1 (d acos = -da / sqrt(1 - a^2)),
    # so the bound is sqrt(2 * 4 ulp(1)) ~ 1e-3 rad at the maximum pixel, 1e-5 elsewhere (a <= 0.999)
    f32 = f.astype(np.complex64)
    p32 = gws.encode(torch.as_tensor(f32, device="cuda"), slm).cpu().numpy()
    ref32 = O.encode(f32.astype(np.complex128))
    d = _circ(p32, ref32)
    a = np.abs(f32) / np.abs(f32).reshape(shape[0], -1).max(1)[:, None, None]
    assert d.max() < 2e-3
    assert d[a < 0.999].max() < 2e-5
    # fixed amplitude scale (clamped above it)
    s = float(np.abs(f32).max() / 3)
    d = _circ(gws.encode(torch.as_tensor(f32, device="cuda"), slm, amp_scale=s).cpu().numpy(),
              O.encode(f32.astype(np.complex128), amp_scale=s))
    assert d.max() < 2e-3


# ---------------------------------------------------------------------------------------
# autotuner, CUDA-graph capture, the batched multi-scene workload
# ---------------------------------------------------------------------------------------

def test_autotune_picks_a_config_and_stays_correct():
    slm = SLM(120, 176, 8e-6, 8e-6, (638e-9, 520e-9, 450e-9))
    sc = surface_scene(30, 300, slm, n_surfaces=3)
    g = dev(sc)
    best = gws.autotune(g, slm)
    assert best in (1, 2, 3, 4, 5)
    u = gws.forward(g, slm, domain=gws.DOMAIN_SPECTRUM).cpu().numpy()  # tile_cfg 0 -> the tuned one
    assert max(per_lambda_rel(u, O.spectrum(sc, slm))) < TOLMX


def test_batched_forward_replays_from_a_cuda_graph():
    slm = SLM(96, 128, 8e-6, 8e-6, (638e-9, 520e-9, 450e-9))
    scenes = [surface_scene(40 + k, n, slm, n_surfaces=2) for k, n in enumerate([200, 35, 1, 120, 0, 64])]
    gs = [dev(s) for s in scenes]
    S = gws.Slm.of(slm)
    gws.prepare(S, n_scenes=len(gs))
    ws = torch.empty(gws.workspace_size([g.n for g in gs], S, gws.make_opts()), dtype=torch.uint8, device="cuda")
    ref = gws.forward_batched(gs, slm, workspace=ws)
    outs = [torch.empty_like(r) for r in ref]
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        gws.forward_batched(gs, slm, outs=outs, workspace=ws)
    torch.cuda.current_stream().wait_stream(side)
    torch.cuda.synchronize()
    for o in outs:
        o.zero_()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        gws.forward_batched(gs, slm, outs=outs, workspace=ws)
    graph.replay()
    torch.cuda.synchronize()
    for o, r in zip(outs, ref):
        assert torch.equal(o, r)
    graph.replay()
    torch.cuda.synchronize()
    for o, r in zip(outs, ref):
        assert torch.equal(o, r)


def test_batched_multi_scene_workload():
    """64 scenes of log-uniform size in [1k, 200k] x 3 wavelengths at 1920x1080 in one call:
    sampled spectra of three scenes vs the oracle, and bit-equality with single calls."""
    from paper_2505_06582_gb300.scenes import batched_scenes
    slm = SLM(1080, 1920, 8e-6, 8e-6, (638e-9, 520e-9, 450e-9))
    scenes = batched_scenes(slm)
    gs = [dev(s) for s in scenes]
    outs = gws.forward_batched(gs, slm, domain=gws.DOMAIN_SPECTRUM)
    for k in (0, 17, 63):
        lam, r, c = _samples(slm, 60, k)
        got = outs[k][torch.as_tensor(lam, dtype=torch.long), torch.as_tensor(r, dtype=torch.long),
                      torch.as_tensor(c, dtype=torch.long)].cpu().numpy()
        ref = O.spectrum_at(scenes[k], slm, lam, r, c)
        assert rel_l2(got, ref) < TOLMX
        single = gws.forward(gs[k], slm, domain=gws.DOMAIN_SPECTRUM)
        assert torch.equal(single, outs[k])


def test_isotropic_point_gaussians():
    # the point-cloud special case (s_u = s_v, no rotation): against the oracle, and unchanged by
    # any rotation about the SLM normal (an isotropic disk has no in-plane orientation)
    slm = SLM(64, 80, 8e-6, 8e-6, (638e-9, 450e-9))
    rng = np.random.default_rng(21)
    n = 40
    mean = np.stack([rng.uniform(-2e-4, 2e-4, n), rng.uniform(-2e-4, 2e-4, n), rng.uniform(1e-3, 4e-3, n)], 1)
    s = rng.uniform(8e-6, 24e-6, n).astype(np.float32)
    quat = np.tile(np.array([1, 0, 0, 0], np.float32), (n, 1))
    amp = rng.uniform(0.2, 1.0, (n, 2)).astype(np.float32)
    opa = rng.uniform(0.2, 1.0, n).astype(np.float32)
    sc = make_scene(mean, quat, np.stack([s, s], 1), opa, amp)
    got = gws.forward(dev(sc), gws.Slm.of(slm)).cpu().numpy()
    want = O.field(sc, slm)
    assert max(per_lambda_rel(got, want)) < TOLMX
    ang = rng.uniform(-np.pi, np.pi, n)
    qz = np.stack([np.cos(ang / 2), 0 * ang, 0 * ang, np.sin(ang / 2)], 1).astype(np.float32)
    rot = gws.forward(dev(make_scene(mean, qz, np.stack([s, s], 1), opa, amp)), gws.Slm.of(slm)).cpu().numpy()
    assert max(per_lambda_rel(rot, got)) < 1e-5


def test_isotropic_points_tab3_shape():
    # 15k isotropic point Gaussians (2 px, no rotation) at 1024x1280, 520 nm: sampled spectrum parity
    # and the forward time (the point-cloud CGH of Tab. 3's comparison takes 2.47 s there)
    slm = SLM(1024, 1280, 8e-6, 8e-6, (520e-9,))
    rng = np.random.default_rng(22)
    n = 15_000
    mean = np.stack([rng.uniform(-0.5, 0.5, n) * slm.W * slm.pitch_x, rng.uniform(-0.5, 0.5, n) * slm.H * slm.pitch_y,
                     rng.uniform(1e-3, 5e-3, n)], 1)
    s = (2 * slm.pitch_x * np.exp(rng.normal(0.0, 0.3, n))).astype(np.float32)
    quat = np.tile(np.array([1, 0, 0, 0], np.float32), (n, 1))
    sc = make_scene(mean, quat, np.stack([s, s], 1), rng.uniform(0.2, 1.0, n).astype(np.float32),
                    rng.uniform(0.2, 1.0, (n, 1)).astype(np.float32))
    g = dev(sc)
    S = gws.Slm.of(slm)
    u = gws.forward(g, S, domain=gws.DOMAIN_SPECTRUM)
    lam, r, c = _samples(slm, 200, 23)
    got = u[torch.as_tensor(lam, dtype=torch.long), torch.as_tensor(r, dtype=torch.long),
            torch.as_tensor(c, dtype=torch.long)].cpu().numpy()
    assert rel_l2(got, O.spectrum_at(sc, slm, lam, r, c)) < TOLMX
    out = gws.forward(g, S)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    gws.forward(g, S, out=out)
    e1.record()
    e1.synchronize()
    print(f"isotropic points, 15k @ 1024x1280 (forward to the field): {e0.elapsed_time(e1):.1f} ms")


def test_precision_at_scale_3840x2160():
    """1M Gaussians on random surfaces at 3840x2160 x 3 wavelengths, 3.74 um pitch: the mixed path
    against the oracle at sampled frequencies (all Gaussians), and against the FP64 GPU path over
    the whole grid for a 2000-Gaussian subset; relative L2 printed per wavelength."""
    sc, slm = config_scene("c2_precision_at_scale")
    g = dev(sc)
    u = gws.forward(g, slm, prec=gws.PREC_MIXED, domain=gws.DOMAIN_SPECTRUM)
    lam, r, c = _samples(slm, 150, 7)
    got = u[torch.as_tensor(lam, dtype=torch.long), torch.as_tensor(r, dtype=torch.long),
            torch.as_tensor(c, dtype=torch.long)].cpu().numpy()
    ref = O.spectrum_at(sc, slm, lam, r, c)
    errs = [rel_l2(got[lam == l], ref[lam == l]) for l in range(slm.n_lambda)]
    print("precision at scale, mixed vs oracle (sampled, 1M):", ["%.2e" % e for e in errs])
    assert max(errs) < TOLMX
    del u
    sub = sc.subset(np.arange(0, sc.n, sc.n // 2000)[:2000])
    gsub = dev(sub)
    um = gws.forward(gsub, slm, prec=gws.PREC_MIXED, domain=gws.DOMAIN_SPECTRUM)
    u64 = gws.forward(gsub, slm, prec=gws.PREC_FP64, domain=gws.DOMAIN_SPECTRUM)
    errs = [(torch.linalg.norm(um[l].to(torch.complex128) - u64[l]) / torch.linalg.norm(u64[l])).item()
            for l in range(slm.n_lambda)]
    print("precision at scale, mixed vs FP64 GPU path (2000 Gaussians, whole grid):", ["%.2e" % e for e in errs])
    assert max(errs) < TOLMX
