"""Benchmark of the Gaussian Wave Splatting hot path on GB300.

Workload: 1M Gaussians on random surfaces (seeded), 1920x1080 SLM, 8 um pitch, 3 wavelengths
(638/520/450 nm).  One step = one pass of the whole hot path over the batch: validation and
precompute, depth sort, footprint binning, the mixed-precision splat (Eq. 10 summed by
Eq. 12), the centred inverse FFT, double-phase encoding and -- when the library provides it
-- the differentiable workload's loss (torch: the field refocused to z = 2, 5, 8 mm by the
angular spectrum method against seeded intensity targets) and the backward splat given that
loss's gradient with respect to the field.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Rank 0 prints ONE JSON line.  Under torchrun every rank runs an independent replica
(the path shards by hologram with no exchange): value = holograms of all ranks / max time.
``--impl reference`` times the FP64 CPU oracle (the reference arm of this project) on a
bounded sample of the same workload, on the host cores.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "holograms/s (1M Gaussians, 1920x1080, 3 λ) fwd & fwd+bwd; Gaussian·freq-px/s"
WORKLOAD = "headline_1m_1080p_3l"
# DRAM bytes (read + write) of one launch of each splat on the headline workload, from
# `ncu --metrics dram__bytes_read.sum,dram__bytes_write.sum` of the kernels as they stand
# (forward: per autotuner configuration, the one the bench's tuner picks)
SPLAT_TRAFFIC_MB = {1: 1592.8}  # configuration 1: 1527.00 MB read + 65.79 MB written (per-tile footprint cull)
BWD_TRAFFIC_MB = 685.8     # 396.52 MB read + 289.29 MB written (per-tile footprint cull)
# Per (Gaussian, frequency) pair: the forward needs ex2, sin and cos on the MUFU (32, 16, 16 per
# SM per clock): 1 / (1/32 + 2/16) = 6.4 pairs/clk/SM; its 14 FP32 lane-ops (8 affine, 2 exponent,
# 1 |g| e, 1 sin/cos prescale, 2 accumulations; the phase is reduced once per (record, thread))
# allow 128 / 14 = 9.1.  The backward adds the gradient products and the 12 moment sums: 30 FP32
# lane-ops per pair (8 affine + 1 for arg G, 2 exponent, 1 prescale, 2 e cos / e sin, 2 |g|
# products, 2 a'/b' products, 12 moments; G enters in polar form, the phase is reduced once per
# (record, column)) -> 128 / 30 = 4.27 pairs/clk/SM, below its MUFU 6.4.
FWD_PAIRS_PER_CLK = 6.4
# A configuration that takes the cos of a fraction f of the pixels on the FP32 pipe (an 11 lane-op
# polynomial with its reduction) needs 1/32 + 1/16 + (1 - f)/16 MUFU cycles and 14 + 11 f FP32
# lane-ops per pair: its bound is the smaller of the two rates.
# A column-step configuration evaluates every second pixel pair as its left neighbour's phase
# factor times one per-record rotation (2 sin/cos per record and thread of 8 pixels) and a
# first-order residual: per pair 1/32 + 1.25/16 MUFU cycles (9.14 pairs/clk/SM) and
# (14 + 18) / 2 = 16 FP32 lane-ops (8.0 pairs/clk/SM, the bound).
FWD_STEP_PAIRS_PER_CLK = min(1.0 / (1.0 / 32 + 1.25 / 16), 128.0 / 16.0)


def fwd_pairs_per_clk(cfg_desc) -> tuple[float, str]:
    f = 0.0
    if cfg_desc and cfg_desc.get("column_step"):
        return FWD_STEP_PAIRS_PER_CLK, ("FP32 bound of the column step (16 FP32 lane-ops per pair; MUFU "
                                        "1/32 + 1.25/16 cycles -> 9.14 pairs/clk/SM)")
    if cfg_desc:
        f = 2.0 * cfg_desc.get("cos_pairs_on_fp32", 0) / cfg_desc["px_per_thread"]
    mufu = 1.0 / (1.0 / 32 + 1.0 / 16 + (1.0 - f) / 16)
    fp32 = 128.0 / (14.0 + 11.0 * f)
    if f == 0.0:
        return FWD_PAIRS_PER_CLK, "MUFU bound (ex2 + sin + cos per pair)"
    which = "MUFU" if mufu <= fp32 else "FP32"
    return min(mufu, fp32), (f"{which} bound with the cos of {f:.2f} of the pixels on the FP32 pipe "
                             f"(MUFU {mufu:.2f}, FP32 {fp32:.2f} pairs/clk/SM)")


BWD_PAIRS_PER_CLK = 128.0 / 30.0
# The generic per-pair counts (minimal formula, per-frequency terms amortised
# over Gaussians): forward 23 FP32 issues + 3 MUFU -> min(128/23, 6.4) = 5.57 pairs/clk/SM; backward
# the same 3 MUFU + 23 recompute + 2 x 14 accumulation lane-ops = 51 -> 128/51 = 2.51 pairs/clk/SM.
FWD_PAIRS_PER_CLK_GENERIC = min(128.0 / 23.0, FWD_PAIRS_PER_CLK)
BWD_PAIRS_PER_CLK_GENERIC = 128.0 / 51.0
FOCAL_PLANES = (2e-3, 5e-3, 8e-3)  # refocus planes of the differentiable workload's loss (m)


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=5)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--n", type=int, default=None, help="override the Gaussian count (testing only)")
    p.add_argument("--workload", default=WORKLOAD,
                   help="named workload of paper_2505_06582_gb300.scenes.CONFIGS (default: the headline)")
    p.add_argument("--prec", default="mixed", choices=["mixed", "fp64"],
                   help="fp64: the plain FP64 comparison path (forward + encode only)")
    p.add_argument("--blend", default="oit", choices=["oit", "sorted", "exact", "partial"],
                   help="oit (Eq. 12, the headline), sorted (depth-sorted T at the centres), exact (Algorithm S2,"
                        " forward + encode only) or partial (one partially coherent frame, Eq. 14, forward + encode"
                        " only)")
    p.add_argument("--pc-l", type=int, default=1, help="partial: degree of the angular kernel's SH")
    p.add_argument("--pc-m", type=int, default=1, help="partial: order of the angular kernel's SH")
    p.add_argument("--traffic-mb", type=float, default=None,
                   help="DRAM bytes per splat launch from an ncu capture of this workload (MB)")
    p.add_argument("--front-end", action="store_true",
                   help="start each step from world-space Gaussians (a 2DGS-OIT style scene with degree-3 SH "
                        "opacity) and run the holographics front end first")
    p.add_argument("--batched", action="store_true",
                   help="the batched workload: 64 scenes of log-uniform size in [1k, 200k] Gaussians x 3 wavelengths "
                        "at 1920x1080, one CUDA-graph-captured gws_forward_batched call per step (forward only)")
    p.add_argument("--seeded-cotangent", action="store_true",
                   help="feed the backward a seeded complex cotangent instead of the refocus loss's gradient")
    p.add_argument("--no-context", action="store_true",
                   help="skip the context rows (plain FP64 path at 20k, the 100k differentiable step, the batched "
                        "64-scene graph replay) timed after the main measurement")
    p.add_argument("--tile-sweep", action="store_true",
                   help="time the forward splat of every autotuner configuration on the workload (3 calls each) and "
                        "print them as one JSON line")
    p.add_argument("--tile-cfgs", default=None,
                   help="--tile-sweep: comma-separated configuration ids to time (default: all)")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--cpu-seconds", type=float, default=15.0)
    return p.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-i", str(self.index),
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None

    def _read(self):
        for ln in self.proc.stdout:
            self.lines.append(ln.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.thread.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[4:8]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def max_over_ranks(ms: float, world: int, dist=None, device=None) -> float:
    """Largest per-rank time (the job takes as long as its slowest replica)."""
    if world <= 1 or dist is None:
        return ms
    import torch
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def aggregate_rate(world: int, ms_per_step: float) -> float:
    """Whole-job holograms/s: every rank produces one hologram per step."""
    return world * 1000.0 / ms_per_step


def cpu_baseline(scene, slm, seconds: float, seed=7, keep_samples=False):
    """FP64 oracle on the host cores: sampled frequencies x all Gaussians, scaled to holograms/s.
    With keep_samples, also returns the sampled (wavelength, row, column, spectrum) arrays."""
    import oracle as O
    threads = O.num_threads()
    rng = np.random.default_rng(seed)
    k = 128
    total_pairs, t_used = 0, 0.0
    samples = []
    while t_used < seconds * 0.5:
        lam = rng.integers(0, slm.n_lambda, k).astype(np.int32)
        r = rng.integers(0, slm.H, k).astype(np.int32)
        c = rng.integers(0, slm.W, k).astype(np.int32)
        t0 = time.perf_counter()
        vals = O.spectrum_at(scene, slm, lam, r, c)
        dt = time.perf_counter() - t0
        total_pairs += k * scene.n
        t_used += dt
        if dt < seconds * 0.1:
            k *= 2
        samples.append((lam, r, c, vals))
    pairs_per_s = total_pairs / t_used
    holo = pairs_per_s / (scene.n * slm.H * slm.W * slm.n_lambda)
    res = {"value": holo, "unit": "holograms/s", "cores": threads, "kind": "oracle",
           "sample": f"{total_pairs // scene.n} sampled (wavelength, frequency) spectrum values over all "
                     f"{scene.n} Gaussians in {t_used:.1f} s ({pairs_per_s:.3g} Gaussian-frequency pairs/s); "
                     f"scaled by N*H*W*L; the inverse DFT (O(HW(H+W)), < 0.1% of the pairs) is not timed"}
    if keep_samples:
        return res, [np.concatenate([x[i] for x in samples]) for i in range(4)]
    return res


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    from paper_2505_06582_gb300.scenes import config_scene
    scene, slm = config_scene(args.workload, n=args.n)
    per = []
    for _ in range(args.warmup):
        cpu_baseline(scene, slm, seconds=2.0)
    for _ in range(args.steps):
        per.append(cpu_baseline(scene, slm, seconds=max(4.0, 60.0 / max(args.steps, 1))))
    v = statistics.median(p["value"] for p in per)
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "holograms/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000.0 / v, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": args.workload, "n_gaussians": scene.n, "H": slm.H, "W": slm.W,
                       "n_lambda": slm.n_lambda, "pitch_m": slm.pitch_x},
            "cpu_baseline": {"kind": "oracle", "cores": per[0]["cores"], "sample": per[0]["sample"], "value": v,
                             "unit": "holograms/s"},
            "e2e": {"value": v, "unit": "holograms/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_ours(args):
    import torch
    import torch.distributed as dist

    from paper_2505_06582_gb300 import gws
    from paper_2505_06582_gb300 import refocus
    from paper_2505_06582_gb300.scenes import config_scene, cotangent

    rank, world, local = dist_env()
    if world > 1 and not dist.is_initialized():
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    scene, slm = config_scene(args.workload, n=args.n)
    S = gws.Slm.of(slm)
    front = None
    if args.front_end:
        # world-space input: the same count, grid and wavelengths; the front end makes the splat's input
        from paper_2505_06582_gb300.scenes import CONFIGS, world_scene
        ws_scene = world_scene(CONFIGS[args.workload]["seed"], scene.n, slm,
                               n_surfaces=CONFIGS[args.workload].get("n_surfaces", 8), volume_frac=0.2)

        def tdev(a, dt):
            return torch.as_tensor(np.ascontiguousarray(a), dtype=dt, device=dev)
        front = dict(world=gws.WorldGaussians(tdev(ws_scene.mean, torch.float64), tdev(ws_scene.quat, torch.float32),
                                              tdev(ws_scene.scale, torch.float32), tdev(ws_scene.amp, torch.float32),
                                              sh_opacity=tdev(ws_scene.sh, torch.float32), sh_degree=3),
                     cam=gws.Camera(ws_scene.view, ws_scene.fx, ws_scene.fy, ws_scene.cx, ws_scene.cy,
                                    gws.PROJ_PERSPECTIVE, 0.1),
                     holo=ws_scene.holo, scene=ws_scene)
        g, valid = gws.holographics(front["world"], front["cam"], front["holo"], compact=False)
        if not bool(valid.bool().all()):
            raise RuntimeError("front-end workload: every Gaussian must stay in view")
        from paper_2505_06582_gb300.scenes import Scene
        scene = Scene(*(getattr(g, k).cpu().numpy() for k in ("mean", "quat", "scale", "opacity", "amp")))
    else:
        g = gws.Gaussians.from_scene(scene, dev)
    fp64 = args.prec == "fp64"
    prec = gws.PREC_FP64 if fp64 else gws.PREC_MIXED
    blend = {"oit": gws.BLEND_OIT, "sorted": gws.BLEND_SORTED_T, "exact": gws.BLEND_EXACT,
             "partial": gws.BLEND_PARTIAL_COHERENT}[args.blend]
    have_bwd = not fp64 and args.blend not in ("exact", "partial")
    pc_kw = dict(pc_l=args.pc_l, pc_m=args.pc_m, pc_seed=1) if args.blend == "partial" else {}
    cot = torch.as_tensor(cotangent(11, slm), device=dev)
    stream = torch.cuda.current_stream(dev)
    flush = torch.empty(512 * 1024 * 1024, dtype=torch.uint8, device=dev)  # > L2 (129 MB)
    gws.prepare(S)
    ws = torch.empty(gws.workspace_size([g.n], S, gws.make_opts(prec=prec, blend=blend, **pc_kw)), dtype=torch.uint8,
                     device=dev)
    # autotune the splat tile on a strided 10% sample of the scene (outside the timed region)
    sub = gws.Gaussians(*(getattr(g, k)[::10].contiguous() for k in ("mean", "quat", "scale", "opacity", "amp")))
    tile_cfg = gws.autotune(sub, S, workspace=ws) if not fp64 else 0
    cfg_desc = gws.tile_configs().get(tile_cfg) if tile_cfg else None
    fwd_per_clk, fwd_basis = fwd_pairs_per_clk(cfg_desc)
    field = torch.empty((S.n_lambda, S.H, S.W), dtype=torch.complex128 if fp64 else torch.complex64, device=dev)
    phase = torch.empty((S.n_lambda, S.H, S.W), dtype=torch.float32, device=dev)
    timers = dict(debug_flags=gws.DEBUG_TIME_KERNELS)

    fe0, fe1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    lo0, lo1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    cur = {"g": g}
    # the differentiable workload's loss: refocus to z = 2, 5, 8 mm, seeded intensity targets (set up once)
    use_loss = have_bwd and not args.seeded_cotangent
    if use_loss:
        Hz = refocus.transfer(slm, FOCAL_PLANES, dev)
        gws.forward(g, S, out=field, workspace=ws, prec=prec, blend=blend, **pc_kw)
        targets = refocus.seeded_targets(4, field, Hz)
        loss_val = torch.zeros((), dtype=torch.float32, device=dev)

    def step(timed_kernels):
        kw = dict(timers) if timed_kernels else {}
        kw["prec"] = prec
        kw["blend"] = blend
        kw.update(pc_kw)
        launches = 0
        t_front = None
        if front is not None:
            fe0.record(stream)
            cur["g"], _ = gws.holographics(front["world"], front["cam"], front["holo"], compact=False)
            fe1.record(stream)
            launches += 1
        g = cur["g"]
        gws.forward(g, S, out=field, workspace=ws, **kw)
        launches += gws.last_launch_count()
        t_splat = gws.kernel_time_ms(gws.TIMER_SPLAT_FWD) if timed_kernels else None
        t_fft = gws.kernel_time_ms(gws.TIMER_FFT) if timed_kernels else None
        # everything of the forward call before the splat and after it but the FFT stage: validation,
        # depth sort, transmittance, footprints and binning, records, the per-pixel table
        t_prep = None
        if timed_kernels:
            t_tot = gws.kernel_time_ms(gws.TIMER_TOTAL)
            t_prep = t_tot - t_splat - t_fft if t_tot > 0 else None
        gws.encode(field, S, out=phase, workspace=ws, **kw)
        launches += gws.last_launch_count()
        t_enc = gws.kernel_time_ms(gws.TIMER_ENCODE) if timed_kernels else None
        t_bwd = t_loss = None
        if have_bwd:
            G = cot
            if use_loss:
                lo0.record(stream)
                L, G = refocus.field_cotangent(field, Hz, targets)
                loss_val.copy_(L)
                lo1.record(stream)
            gws.backward(g, S, G, workspace=ws, **kw)
            launches += gws.last_launch_count()
            t_bwd = gws.kernel_time_ms(gws.TIMER_SPLAT_BWD) if timed_kernels else None
            if use_loss and timed_kernels:
                lo1.synchronize()
                t_loss = lo0.elapsed_time(lo1)
        if front is not None and timed_kernels:
            fe1.synchronize()
            t_front = fe0.elapsed_time(fe1)
        return launches, t_splat, t_fft, t_enc, t_bwd, t_front, t_prep, t_loss

    step(False)
    torch.cuda.synchronize()
    for _ in range(args.warmup):
        step(False)
    torch.cuda.synchronize()

    # device-timed steps (inputs resident in HBM; L2 flushed before each step, outside the events)
    clocks = ClockSampler(local)
    clocks.start()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    times, splat_ms, fft_ms, enc_ms, bwd_ms, front_ms, prep_ms, loss_ms, launches = [], [], [], [], [], [], [], [], 0
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    for _ in range(args.steps):
        flush.zero_()
        e0.record(stream)
        n_l, ts, tf, te, tb, tfe, tp, tl = step(True)
        prep_ms.append(tp)
        if tl is not None:
            loss_ms.append(tl)
        if tfe is not None:
            front_ms.append(tfe)
        e1.record(stream)
        e1.synchronize()
        times.append(e0.elapsed_time(e1))
        launches += n_l
        splat_ms.append(ts)
        fft_ms.append(tf)
        enc_ms.append(te)
        if tb is not None:
            bwd_ms.append(tb)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    clk = clocks.stop()
    ms = max_over_ranks(sum(times) / len(times), world, dist if world > 1 else None, dev)
    value = aggregate_rate(world, ms)

    # end to end through the public API with host buffers (pinned), copies inside the timed region
    src = front["world"] if front is not None else g
    in_keys = ("mean", "quat", "scale", "sh_opacity", "amp") if front is not None else \
        ("mean", "quat", "scale", "opacity", "amp")
    host = {k: getattr(src, k).cpu().pin_memory() for k in in_keys}
    cot_host = cot.cpu().pin_memory()
    tgt_host = targets.cpu().pin_memory() if use_loss else None
    tbuf = torch.empty_like(targets) if use_loss else None
    loss_host = torch.empty((), dtype=torch.float32).pin_memory()
    phase_host = torch.empty(phase.shape, dtype=phase.dtype).pin_memory()
    dbuf = {k: torch.empty_like(getattr(src, k)) for k in host}
    cbuf = torch.empty_like(cot)
    grads_host = {k: torch.empty(getattr(g, k).shape, dtype=getattr(g, k).dtype).pin_memory()
                  for k in ("mean", "quat", "scale", "opacity", "amp")}
    h2d = sum(v.numel() * v.element_size() for v in host.values())
    if have_bwd:  # the step's other input: the loss's targets (or the seeded cotangent)
        h2d += tgt_host.numel() * tgt_host.element_size() if use_loss else cot_host.numel() * cot_host.element_size()
    d2h = phase_host.numel() * phase_host.element_size() + (
        sum(v.numel() * v.element_size() for v in grads_host.values()) + (4 if use_loss else 0) if have_bwd else 0)
    e2e_times = []
    for _ in range(max(2, min(args.steps, 3))):
        flush.zero_()
        torch.cuda.synchronize()
        e0.record(stream)
        for k in host:
            dbuf[k].copy_(host[k], non_blocking=True)
        if front is not None:
            wd = gws.WorldGaussians(dbuf["mean"], dbuf["quat"], dbuf["scale"], dbuf["amp"],
                                    sh_opacity=dbuf["sh_opacity"], sh_degree=3)
            gd, _ = gws.holographics(wd, front["cam"], front["holo"], compact=False)
        else:
            gd = gws.Gaussians(dbuf["mean"], dbuf["quat"], dbuf["scale"], dbuf["opacity"], dbuf["amp"])
        gws.forward(gd, S, out=field, workspace=ws, prec=prec, blend=blend, **pc_kw)
        gws.encode(field, S, out=phase, workspace=ws)
        phase_host.copy_(phase, non_blocking=True)
        if have_bwd:
            if use_loss:
                tbuf.copy_(tgt_host, non_blocking=True)
                L, Gd = refocus.field_cotangent(field, Hz, tbuf)
                loss_host.copy_(L, non_blocking=True)
            else:
                cbuf.copy_(cot_host, non_blocking=True)
                Gd = cbuf
            gr = gws.backward(gd, S, Gd, workspace=ws, blend=blend)
            for k in grads_host:
                grads_host[k].copy_(gr[k], non_blocking=True)
        e1.record(stream)
        e1.synchronize()
        e2e_times.append(e0.elapsed_time(e1))
    e2e_ms = max_over_ranks(statistics.median(e2e_times), world, dist if world > 1 else None, dev)

    # rooflines of the two splats: algorithmic pairs (the footprint pairs both visit) / event time
    dense = g.n * S.H * S.W * S.n_lambda
    pairs = dense if fp64 else gws.footprint_pairs(g, S, workspace=ws)
    splat = statistics.median(splat_ms)
    sm_mhz = clk.get("sm_mhz") or 1440.0
    n_sm = torch.cuda.get_device_properties(dev).multi_processor_count
    dom_ms = {"splat_fwd": splat, "fft": statistics.median(fft_ms), "encode": statistics.median(enc_ms)}
    if all(t is not None for t in prep_ms):
        dom_ms["prep"] = statistics.median(prep_ms)
    if bwd_ms:
        dom_ms["splat_bwd"] = statistics.median(bwd_ms)
    if loss_ms:
        dom_ms["refocus_loss"] = statistics.median(loss_ms)
    full_size = args.workload == WORKLOAD and not fp64 and args.n is None and args.blend == "oit"

    def roof(kernel, kms, per_clk, basis, traffic_mb, generic_per_clk=None, generic_basis=""):
        achieved = pairs / (kms * 1e-3)
        peak = n_sm * sm_mhz * 1e6 * per_clk
        r = {"kernel": kernel, "bound": "alu", "achieved": achieved / 1e9, "peak": peak / 1e9, "unit": "Gpair/s",
             "frac": achieved / peak, "traffic": None if traffic_mb is None else traffic_mb * 1e6,
             "peak_basis": f"{n_sm} SMs x {sm_mhz:.0f} MHz (median sampled) x {per_clk:.2f} pairs/clk/SM, " + basis}
        if generic_per_clk is not None:
            sp = n_sm * sm_mhz * 1e6 * generic_per_clk
            r["generic_count"] = {"peak": sp / 1e9, "frac": achieved / sp, "per_clk": generic_per_clk,
                                 "basis": generic_basis}
        return r

    if args.blend in ("exact", "partial"):
        # the batch loop (one-Gaussian spectra, batched inverse FFT, mask or kernel product, batched
        # forward FFT, accumulation) moves each (Gaussian, wavelength, pixel) value 8 times at 8 B:
        # spectra write, inverse FFT read + write, mask read + write, forward FFT read + write,
        # accumulation read; cuFFT's internal passes are not counted
        hbm_pk = 6785.9
        try:
            hbm_pk = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))["hbm_gbs"]
        except (OSError, KeyError, ValueError):
            pass
        lb = 64.0 * g.n * S.H * S.W * S.n_lambda
        ach = lb / (splat * 1e-3) / 1e9
        rooflines = {"splat_fwd": {"kernel": "batch loop (k_single_spectra, cuFFT, k_exact_mask / k_pc_apply, "
                                             "k_exact_accum)", "bound": "hbm", "achieved": ach, "peak": hbm_pk,
                                   "unit": "GB/s", "frac": ach / hbm_pk, "traffic": None,
                                   "note": "64 algorithmic bytes per (Gaussian, wavelength, pixel)"}}
    else:
        rooflines = {"splat_fwd": roof(
            "k_splat_fp64" if fp64 else "k_splat_mixed", splat, fwd_per_clk,
            fwd_basis + (" (FP32/MUFU peak; the FP64 path runs on the FP64 pipe)" if fp64 else ""),
            args.traffic_mb if args.traffic_mb is not None else (SPLAT_TRAFFIC_MB.get(tile_cfg) if full_size else None),
            None if fp64 else FWD_PAIRS_PER_CLK_GENERIC,
            "generic count: 23 FP32 issues + 3 MUFU per pair -> min(128/23, 6.4) pairs/clk/SM")}
    if bwd_ms:
        rooflines["splat_bwd"] = roof("k_splat_bwd", dom_ms["splat_bwd"], BWD_PAIRS_PER_CLK,
                                      "FP32 bound (30 lane-ops per pair at 128 lanes/clk/SM; MUFU bound 6.4)",
                                      BWD_TRAFFIC_MB if full_size else None, BWD_PAIRS_PER_CLK_GENERIC,
                                      "generic count: 3 MUFU + 23 recompute + 2 x 14 accumulation = 51 FP32 lane-ops "
                                      "per pair -> 128/51 pairs/clk/SM")
    if front_ms:
        dom_ms["front_end"] = statistics.median(front_ms)
        # algorithmic bytes per Gaussian: mean 24 + quat 16 + scale 12 + 16 SH floats 64 read,
        # mean 24 + quat 16 + scale 8 + opacity 4 + flag 1 written
        fb = 169 * g.n
        hbm_peak_fe = 6785.9
        try:
            hbm_peak_fe = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))["hbm_gbs"]
        except (OSError, KeyError, ValueError):
            pass
        ach = fb / (dom_ms["front_end"] * 1e-3) / 1e9
        rooflines["front_end"] = {"kernel": "k_holographics", "bound": "hbm", "achieved": ach, "peak": hbm_peak_fe,
                                  "unit": "GB/s", "frac": ach / hbm_peak_fe, "traffic": None,
                                  "note": "169 algorithmic bytes per Gaussian; the FP64 per-Gaussian algebra, not "
                                          "HBM, sets its time"}
    dominant = max((k for k in rooflines if k != "front_end"), key=lambda k: dom_ms[k])
    fwd_ms = ms - (dom_ms.get("splat_bwd", 0.0))
    # HBM-bound stages: algorithmic bytes = one read + one write of every slice per pass
    hbm_peak = 6785.9
    try:
        hbm_peak = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))["hbm_gbs"]
    except (OSError, KeyError, ValueError):
        pass
    cplx = 16 if fp64 else 8
    px = S.H * S.W * S.n_lambda
    fft_bytes = 2 * 2 * cplx * px  # in-place inverse FFT (read + write) + post-modulation (read + write)
    enc_bytes = cplx * px + (cplx + 4) * px  # max-|u| pass (read) + encoding (read field, write phase)
    hbm = {"fft_stage": {"bytes": fft_bytes, "ms": dom_ms["fft"],
                         "achieved_gbs": fft_bytes / (dom_ms["fft"] * 1e-3) / 1e9},
           "encode": {"bytes": enc_bytes, "ms": dom_ms["encode"],
                      "achieved_gbs": enc_bytes / (dom_ms["encode"] * 1e-3) / 1e9}}
    for v in hbm.values():
        v["peak_gbs"] = hbm_peak
        v["frac"] = v["achieved_gbs"] / hbm_peak

    line = {"metric": METRIC, "value": value, "unit": "holograms/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
            "config": {"workload": args.workload + ("+front_end(world_scene)" if front is not None else ""),
                       "n_gaussians": g.n, "H": S.H, "W": S.W, "n_lambda": S.n_lambda,
                       "pitch_m": S.pitch_x, "blend": args.blend, "precision": args.prec,
                       "trunc_eps": None if fp64 else 1e-5,
                       "step": ("front_end+" if front is not None else "") + "forward+encode"
                               + (("+refocus_loss(z=2,5,8mm)" if use_loss else "+seeded_cotangent") + "+backward"
                                  if have_bwd else ""), "tile_cfg": tile_cfg, "tile_cfg_desc": cfg_desc,
                       "l2": "flushed before each timed step (512 MB write)", "parallelism": f"replicas x{world}"},
            "fwd_holograms_per_s": world * 1000.0 / fwd_ms if have_bwd else value,
            "pairs": {"dense_per_hologram": dense, "algorithmic_per_hologram": pairs,
                      "dense_pairs_per_s": world * dense / (fwd_ms * 1e-3),
                      "algorithmic_pairs_per_s": world * pairs / (fwd_ms * 1e-3)},
            "kernel_ms": dom_ms,
            "roofline": rooflines[dominant],
            "rooflines": rooflines,
            "hbm": hbm,
            "e2e": {"value": aggregate_rate(world, e2e_ms), "unit": "holograms/s", "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": d2h},
            "gpu_launches": launches,
            "clocks": clk}
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"], smp = cpu_baseline(scene, slm, args.cpu_seconds, keep_samples=True)
        # parity of this workload's spectrum against the oracle values the baseline just computed (one
        # more forward, outside the timed region): rel-L2 per wavelength over the sampled frequencies
        spec = gws.forward(g, S, workspace=ws, prec=prec, blend=blend, domain=gws.DOMAIN_SPECTRUM, **pc_kw)
        lam_i, r_i, c_i, ref = smp
        got = spec[torch.as_tensor(lam_i.astype(np.int64), device=dev), torch.as_tensor(r_i.astype(np.int64), device=dev),
                   torch.as_tensor(c_i.astype(np.int64), device=dev)].cpu().numpy().astype(np.complex128)
        per = []
        for l in range(S.n_lambda):
            m = lam_i == l
            per.append(float(np.linalg.norm(got[m] - ref[m]) / max(np.linalg.norm(ref[m]), 1e-300)) if m.any() else None)
        line["parity"] = {"rel_l2_per_lambda": per, "wavelengths_nm": [round(w * 1e9, 1) for w in slm.wavelengths],
                          "samples": int(lam_i.size), "against": "FP64 oracle (gwso_spectrum_at), same samples as "
                          "cpu_baseline", "tolerance": 1e-6 if fp64 else 2e-4, "domain": "spectrum"}
        del spec
    if rank == 0 and world == 1 and not args.no_context and args.workload == WORKLOAD and args.n is None \
            and not fp64 and args.blend == "oit" and front is None:
        del ws
        torch.cuda.empty_cache()
        line["context"] = run_context(dev)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def _event_ms(fn, stream, flush=None):
    """CUDA-event time of fn() on the stream (L2 flushed first when a flush buffer is given)."""
    import torch
    if flush is not None:
        flush.zero_()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    fn()
    e1.record(stream)
    e1.synchronize()
    return e0.elapsed_time(e1)


def run_context(dev):
    """One step each of the other workloads, timed in the same run (rank 0, after the headline):
    the plain FP64 GPU path next to the mixed path at 20k Gaussians (1920x1080, 3 wavelengths), the
    100k differentiable step (forward + encode + refocus loss + backward), the 1M-Gaussian forward at
    3840x2160 and one CUDA-graph replay of the batched 64-scene forward."""
    import torch

    from paper_2505_06582_gb300 import gws, refocus
    from paper_2505_06582_gb300.scenes import config_scene

    stream = torch.cuda.current_stream(dev)
    flush = torch.empty(512 * 1024 * 1024, dtype=torch.uint8, device=dev)
    out = {}
    # plain FP64 GPU path vs the mixed path at 20k Gaussians
    sc, slm = config_scene("c1_slm_size")
    S = gws.Slm.of(slm)
    g = gws.Gaussians.from_scene(sc, dev)
    ws = torch.empty(max(gws.workspace_size([g.n], S, gws.make_opts(prec=p)) for p in (gws.PREC_FP64, gws.PREC_MIXED)),
                     dtype=torch.uint8, device=dev)
    f64 = torch.empty((S.n_lambda, S.H, S.W), dtype=torch.complex128, device=dev)
    fmx = torch.empty((S.n_lambda, S.H, S.W), dtype=torch.complex64, device=dev)
    small = gws.Gaussians(*(getattr(g, k)[:64].contiguous() for k in ("mean", "quat", "scale", "opacity", "amp")))
    gws.forward(small, S, out=f64, workspace=ws, prec=gws.PREC_FP64)  # module and plan warm-up
    for _ in range(2):
        gws.forward(g, S, out=fmx, workspace=ws, prec=gws.PREC_MIXED)
    t_mx = _event_ms(lambda: gws.forward(g, S, out=fmx, workspace=ws, prec=gws.PREC_MIXED), stream, flush)
    t_64 = _event_ms(lambda: gws.forward(g, S, out=f64, workspace=ws, prec=gws.PREC_FP64), stream, flush)
    a, b = f64.cpu().numpy(), fmx.cpu().numpy().astype(np.complex128)
    rel = [float(np.linalg.norm(b[l] - a[l]) / np.linalg.norm(a[l])) for l in range(S.n_lambda)]
    dense = g.n * S.H * S.W * S.n_lambda
    out["c1_20k_fp64_vs_mixed"] = {
        "workload": "c1_slm_size: 20k Gaussians, 1920x1080, 3 wavelengths, forward (splat + inverse DFT)",
        "fp64_ms": t_64, "mixed_ms": t_mx, "fp64_dense_pairs_per_s": dense / (t_64 * 1e-3),
        "mixed_dense_pairs_per_s": dense / (t_mx * 1e-3), "speedup_mixed_over_fp64": t_64 / t_mx,
        "mixed_vs_fp64_rel_l2_per_lambda": rel, "l2": "flushed before each call"}
    del f64, fmx, ws, g
    torch.cuda.empty_cache()
    # the differentiable workload, one step
    sc, slm = config_scene("c4_differentiable")
    S = gws.Slm.of(slm)
    g = gws.Gaussians.from_scene(sc, dev)
    ws = torch.empty(gws.workspace_size([g.n], S, gws.make_opts()), dtype=torch.uint8, device=dev)
    field = torch.empty((S.n_lambda, S.H, S.W), dtype=torch.complex64, device=dev)
    phase = torch.empty((S.n_lambda, S.H, S.W), dtype=torch.float32, device=dev)
    Hz = refocus.transfer(slm, FOCAL_PLANES, dev)
    gws.forward(g, S, out=field, workspace=ws)
    targets = refocus.seeded_targets(4, field, Hz)

    def c4_step():
        gws.forward(g, S, out=field, workspace=ws)
        gws.encode(field, S, out=phase, workspace=ws)
        _, G = refocus.field_cotangent(field, Hz, targets)
        gws.backward(g, S, G, workspace=ws)

    for _ in range(2):
        c4_step()
    t_c4 = statistics.median(_event_ms(c4_step, stream, flush) for _ in range(3))
    out["c4_differentiable_step"] = {
        "workload": "c4_differentiable: 100k Gaussians, 1920x1080, 3 wavelengths; forward + encode + refocus loss "
                    "(z = 2, 5, 8 mm) + backward", "ms": t_c4, "holograms_per_s": 1000.0 / t_c4,
        "l2": "flushed before each step"}
    del field, phase, ws, g, Hz, targets
    torch.cuda.empty_cache()
    # precision at scale: 1M Gaussians at 3840x2160, 3.74 um pitch, the mixed forward (its parity per
    # frequency band against the oracle is a GPU test, not part of this timing)
    sc, slm = config_scene("c2_precision_at_scale")
    S = gws.Slm.of(slm)
    g = gws.Gaussians.from_scene(sc, dev)
    ws = torch.empty(gws.workspace_size([g.n], S, gws.make_opts()), dtype=torch.uint8, device=dev)
    field = torch.empty((S.n_lambda, S.H, S.W), dtype=torch.complex64, device=dev)
    gws.forward(g, S, out=field, workspace=ws)
    t_c2 = _event_ms(lambda: gws.forward(g, S, out=field, workspace=ws), stream, flush)
    pairs_c2 = gws.footprint_pairs(g, S, workspace=ws)
    out["c2_precision_at_scale"] = {
        "workload": "c2_precision_at_scale: 1M Gaussians, 3840x2160, 3.74 um pitch, 3 wavelengths; mixed forward "
                    "(splat + inverse DFT)", "ms": t_c2, "holograms_per_s": 1000.0 / t_c2,
        "algorithmic_pairs_per_s": pairs_c2 / (t_c2 * 1e-3),
        "parity": "tests/test_gpu_forward.py::test_full_size_band_stratified_spectrum[c2_precision_at_scale]",
        "l2": "flushed before the call"}
    del field, ws, g
    torch.cuda.empty_cache()
    # the batched workload: one graph replay
    t_b, pairs_b, n_scenes, n_tot, _ = batched_graph_ms(dev, warmup=1, steps=1, flush=flush)
    out["c3_batched_graph"] = {
        "workload": f"batched: {n_scenes} scenes of log-uniform [1k, 200k] Gaussians ({n_tot} in all) x 3 "
                    "wavelengths, 1920x1080, one CUDA-graph replay of gws_forward_batched", "ms": t_b,
        "holograms_per_s": n_scenes * 1000.0 / t_b, "algorithmic_pairs_per_s": pairs_b / (t_b * 1e-3),
        "l2": "flushed before the replay"}
    return out


def batched_graph_ms(dev, warmup, steps, flush=None):
    """Times graph replays of gws_forward_batched on the 64-scene workload: (median ms, footprint pairs,
    scenes, Gaussians, kernel launches per replay)."""
    import torch

    from paper_2505_06582_gb300 import gws
    from paper_2505_06582_gb300.scenes import SLM, batched_scenes

    slm = SLM(1080, 1920, 8e-6, 8e-6, (638e-9, 520e-9, 450e-9))
    scenes = batched_scenes(slm)
    gs = [gws.Gaussians.from_scene(sc, dev) for sc in scenes]
    S = gws.Slm.of(slm)
    gws.prepare(S, n_scenes=len(gs))
    ws = torch.empty(gws.workspace_size([g.n for g in gs], S, gws.make_opts()), dtype=torch.uint8, device=dev)
    outs = [torch.empty((S.n_lambda, S.H, S.W), dtype=torch.complex64, device=dev) for _ in gs]
    side = torch.cuda.Stream(dev)
    side.wait_stream(torch.cuda.current_stream(dev))
    with torch.cuda.stream(side):
        gws.forward_batched(gs, S, outs=outs, workspace=ws)
    torch.cuda.current_stream(dev).wait_stream(side)
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        gws.forward_batched(gs, S, outs=outs, workspace=ws)
    launches = gws.last_launch_count()
    if flush is None:
        flush = torch.empty(512 * 1024 * 1024, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream(dev)
    for _ in range(warmup):
        graph.replay()
    torch.cuda.synchronize()
    times = [_event_ms(graph.replay, stream, flush) for _ in range(steps)]
    pairs = sum(gws.footprint_pairs(g, S, workspace=ws) for g in gs)
    n_tot = sum(g.n for g in gs)
    del graph, outs, ws
    return statistics.median(times), pairs, len(gs), n_tot, launches


def run_batched(args):
    """64 scenes x 3 wavelengths in one persistent splat launch, captured in a CUDA graph and replayed
    once per step (forward: splat + inverse FFTs); holograms/s = 64 / step time."""
    import torch

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    clocks = ClockSampler(local)
    clocks.start()
    ms, pairs, n_scenes, n_tot, launches = batched_graph_ms(dev, warmup=max(args.warmup, 3), steps=args.steps)
    clk = clocks.stop()
    sm_mhz = clk.get("sm_mhz") or 1440.0
    n_sm = torch.cuda.get_device_properties(dev).multi_processor_count
    peak = n_sm * sm_mhz * 1e6 * FWD_PAIRS_PER_CLK
    ach = pairs / (ms * 1e-3)
    line = {"metric": METRIC, "value": n_scenes * 1000.0 / ms, "unit": "holograms/s", "n_gpus": 1,
            "steps": args.steps, "warmup": max(args.warmup, 3), "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
            "config": {"workload": "batched_64_scenes_1k_200k_1080p_3l", "n_scenes": n_scenes,
                       "n_gaussians": n_tot, "H": 1080, "W": 1920, "n_lambda": 3,
                       "step": "one graph replay of gws_forward_batched (splat + inverse FFTs)",
                       "l2": "flushed before each timed step (512 MB write)", "parallelism": "single GPU"},
            "roofline": {"kernel": "k_splat_mixed (whole graph timed)", "bound": "alu", "achieved": ach / 1e9,
                         "peak": peak / 1e9, "unit": "Gpair/s", "frac": ach / peak, "traffic": None,
                         "peak_basis": f"{n_sm} SMs x {sm_mhz:.0f} MHz x {FWD_PAIRS_PER_CLK} pairs/clk/SM (MUFU)"},
            "gpu_launches": launches, "clocks": clk}
    print(json.dumps(line), flush=True)


def run_tile_sweep(args):
    """Forward splat time of every configuration of the autotuner's search space on the workload."""
    import torch

    from paper_2505_06582_gb300 import gws
    from paper_2505_06582_gb300.scenes import config_scene

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    scene, slm = config_scene(args.workload, n=args.n)
    S = gws.Slm.of(slm)
    g = gws.Gaussians.from_scene(scene, dev)
    ws = torch.empty(gws.workspace_size([g.n], S, gws.make_opts()), dtype=torch.uint8, device=dev)
    out = torch.empty((S.n_lambda, S.H, S.W), dtype=torch.complex64, device=dev)
    gws.prepare(S)
    clocks = ClockSampler(local)
    clocks.start()
    rows = []
    only = {int(x) for x in args.tile_cfgs.split(",")} if args.tile_cfgs else None
    for c, d in gws.tile_configs().items():
        if only is not None and c not in only:
            continue
        ts = []
        for _ in range(3):
            gws.forward(g, S, out=out, workspace=ws, tile_cfg=c, domain=gws.DOMAIN_SPECTRUM,
                        debug_flags=gws.DEBUG_TIME_KERNELS)
            ts.append(gws.kernel_time_ms(gws.TIMER_SPLAT_FWD))
        rows.append(dict(d, id=c, splat_ms=statistics.median(ts)))
    clk = clocks.stop()
    if rank == 0:
        print(json.dumps({"mode": "tile_sweep", "workload": args.workload, "n_gaussians": g.n,
                          "configs": rows, "clocks": clk}), flush=True)


def main():
    args = parse()
    if args.tile_sweep:
        run_tile_sweep(args)
    elif args.impl == "reference":
        run_reference(args)
    elif args.batched:
        run_batched(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
