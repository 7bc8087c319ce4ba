"""Benchmark: Lenia cell-updates/s on one GB300 (or N independent replicas).

Workload: the 2048 x 2048, 3-channel, 15-kernel (R = 18) world with
localized mu/sigma gene maps and gene maintenance on (seeded synthetic
input shaped like the paper's runs: 16 genotype patches whose genes are
matched to their noise, so the patch interiors pass every kernel's growth
test).  One step = one pass of the whole hot path: row FFTs, column FFT x
kernel spectra x inverse, inverse row FFTs, diffusion + growth + alpha mask
+ clipped update, and per-channel stats.  Every timed step advances the same
live state by one step (inputs 551 MB, larger than L2).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

With --gpus N > 1 and no torchrun environment the script starts N ranks
itself (torch.distributed.run on 127.0.0.1), one replica world per GPU.

Prints one JSON line (rank 0): the step's throughput, the dominant kernel's
HBM roofline (with its ncu DRAM traffic), the FFT passes against the
measured FP32 peak, an end-to-end serving loop through host buffers, clocks
sampled during the timed region, the CPU oracle baseline, and (N = 1) the
adjoint, batched-world, evolution, ring and small-world legs (--leg NAME
runs one alone).  --impl reference times the FP64 CPU oracle on the host
cores over a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "cell-updates/s at 2048^2 FP32 (% HBM roofline); batched & adjoint vs plain step"
UNIT = "cell-updates/s"
WORKLOAD = ("lenia 2048x2048, 3 channels, 15 shell kernels R=18, localized mu/sigma maps (16 genotype "
            "patches matched to their noise), gene maintenance")
# Algorithmic bytes per site-step: A read + write (3 channels x 4 B x 2) and
# the 30 gene planes read + write (30 x 4 B x 2).
ALG_BYTES_PER_SITE = 3 * 4 * 2 + 30 * 4 * 2


def fft_flops(H, W, C, K):
    """Flops of the FFT route per step, counted the standard way (a complex
    FFT of n points 5 n log2 n, a real one half that): C forward real 2D
    transforms; per kernel the spectral product (a real factor on W/2 + 1
    columns) and one inverse real 2D transform."""
    lw, lh = math.log2(W), math.log2(H)
    rows = H * 2.5 * W * lw                     # real row transforms of one plane
    cols = (W // 2 + 1) * 5.0 * H * lh          # complex column transforms of one half spectrum
    return C * (rows + cols) + K * ((W // 2 + 1) * H * 2.0 + cols + rows)


def _traffic(kernel: str, name="epilogue_traffic.json", key="dram_bytes_per_launch"):
    """DRAM bytes (per launch of `kernel`, or per step) from a committed ncu
    capture, or None when the sources changed since the capture."""
    import hashlib
    try:
        with open(os.path.join(ROOT, "profiles", name)) as f:
            d = json.load(f)
        if d.get("kernel") != kernel:
            return None
        h = hashlib.sha256()
        for src in d["sources"]:
            with open(os.path.join(ROOT, src), "rb") as f:
                h.update(f.read())
        return int(d[key]) if h.hexdigest() == d["sources_sha256"] else None
    except (OSError, KeyError, ValueError):
        return None


def _bf16_peak():
    """Measured dense BF16 tensor peak in TFLOP/s (burst), or the fallback."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["bf16_tflops"])
    except Exception:
        return 1900.0


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class Clocks:
    """nvidia-smi sampling during the timed region."""

    def __init__(self, index: int):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--id={index}", f"--query-gpu={q}",
                                       "--format=csv,noheader,nounits", "-lms", "100"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except (FileNotFoundError, OSError):
            self.p = None

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.p.kill()
        self.f.flush()
        self.f.seek(0)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.f:
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        os.unlink(self.f.name)
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": float(max(mx)) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def fp32_line(prof, H, W, scalar_tflops, pair_tflops):
    """FP32-pipe fraction of the FFT passes (arithmetic- and latency-bound,
    not DRAM-bound) against the measured FMA peak."""
    names = ("rows_r2c", "cols_conv", "rows_c2r")
    ms = sum(prof[k][0] / max(1, prof[k][1]) for k in names if k in prof)
    flops = fft_flops(H, W, 3, 15)
    peak = max(scalar_tflops, pair_tflops)
    achieved = flops / (ms / 1e3) / 1e12 if ms > 0 else 0.0
    return {"peak_tflops": peak, "peak_kind": "measured (FMA chains on every SM)",
            "peak_scalar_tflops": scalar_tflops, "peak_pair_tflops": pair_tflops,
            "fft_passes": {"kernels": list(names), "flop_per_site": flops / (H * W), "ms": ms,
                           "achieved_tflops": achieved, "frac": achieved / peak if peak > 0 else None}}


def cufft_yardstick(torch, lenia, ctx, world, stream, ours_ms, reps=20):
    """The same convolutions through torch.fft (cuFFT) as a timing yardstick
    (not a path of the library): rfft2 of the C channel planes, the product
    of each kernel's real spectrum with its source channel's spectrum, and
    irfft2 of the K products -- the transforms the three FFT passes perform
    (the products are one extra elementwise pass here)."""
    H, W = world.height, world.width
    dev = torch.device("cuda")
    spec = []
    for k, kd in enumerate(world.kernels):
        R = kd.radius
        w = torch.from_numpy(lenia.lenia_kernel_weights(ctx, k, R)).to(dev, torch.float32)
        full = torch.zeros((H, W), dtype=torch.float32, device=dev)
        idx = torch.arange(-R, R + 1, device=dev)
        full[(idx[:, None] % H), (idx[None, :] % W)] = w          # correlation taps at (dy, dx)
        spec.append(torch.fft.rfft2(full).conj())
    S = torch.stack(spec)
    src = torch.tensor([k.src for k in world.kernels], device=dev)
    A = torch.from_numpy(world.A).to(dev)

    def run():
        F = torch.fft.rfft2(A)
        return torch.fft.irfft2(F[src] * S, s=(H, W))
    for _ in range(3):
        U = run()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        U = run()
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / reps
    del U, S, A
    return {"cufft_ms": ms, "ours_ms": ours_ms, "ours_over_cufft_time": ours_ms / ms if ms > 0 else None,
            "note": "torch.fft (cuFFT): rfft2 of 3 planes, 15 spectral products, irfft2 of 15 planes, on "
                    "torch's current stream; ours: the r2c, column and c2r passes of the same step"}


def workload_config(ws, size=2048):
    """The benchmark workload, named by what it is (both arms print the same
    object; other sizes are profiling runs of the same recipe).  How an arm
    computes it (its convolution path) goes beside the config, not in it."""
    return {"workload": WORKLOAD if size == 2048 else WORKLOAD.replace("2048x2048", f"{size}x{size}"),
            "height": size, "width": size, "channels": 3, "kernels": 15, "radius": 18,
            "gene_planes": 30, "worlds": ws, "parallelism": "replicas" if ws > 1 else "single",
            "l2": "inputs larger than L2 (A + P = 551 MB per world)",
            "state": "each timed step advances the same live state (A0, P0) by one step"}


def adjoint_leg(torch, lenia, inputs, stream):
    """Forward rollout vs rollout adjoint: 256^2, 3 channels, 15 kernels R=13,
    global genes, 64 steps, checkpoints every 8; and the same with every state
    kept (checkpoint every step: the reverse pass recomputes nothing)."""
    w = inputs.global_multi_channel()
    n = 64
    out = {"workload": "256x256, 3 channels, 15 kernels R=13, global genes, 64 steps, checkpoint every 8"}
    for ck in (8, 1):
        cfg, ks = lenia.config_from_world(w, lenia.CONV_AUTO, max_rollout_steps=n, ckpt_every=ck)
        ctx = lenia.lenia_init(cfg, ks, stream)
        try:
            A0 = torch.from_numpy(w.A).cuda()
            A = A0.clone()
            gA_T = torch.ones_like(A0)
            gA0 = torch.empty_like(A0)
            gg = torch.empty((w.n_kernels, 3), dtype=torch.float32, device="cuda")
            ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
            for _ in range(2):                                   # warm-up
                A.copy_(A0)
                lenia.lenia_rollout(ctx, A, None, n, None, stream)
                lenia.lenia_backward(ctx, A0, None, n, gA_T, gA0, gg, stream)
            reps = 5
            torch.cuda.synchronize()
            ev[0].record(stream)
            for _ in range(reps):
                A.copy_(A0)
                lenia.lenia_rollout(ctx, A, None, n, None, stream)
            ev[1].record(stream)
            for _ in range(reps):
                lenia.lenia_backward(ctx, A0, None, n, gA_T, gA0, gg, stream)
            ev[2].record(stream)
            torch.cuda.synchronize()
            lenia.lenia_check(ctx)
            fwd = ev[0].elapsed_time(ev[1]) / reps
            bwd = ev[1].elapsed_time(ev[2]) / reps
            path = "fft" if lenia.lenia_conv_path(ctx) == lenia.CONV_FFT else "direct"
        finally:
            lenia.lenia_destroy(ctx)
        if ck == 8:
            out.update({"fwd_ms": fwd, "bwd_ms": bwd, "fwd_plus_bwd_over_fwd": (fwd + bwd) / fwd,
                        "conv_path": path,
                        "note": "bwd recomputes the forward from checkpoints inside lenia_backward"})
        else:
            out["every_state_kept"] = {"fwd_ms": fwd, "bwd_ms": bwd, "fwd_plus_bwd_over_fwd": (fwd + bwd) / fwd,
                                       "note": "checkpoint every step: the forward pass inside lenia_backward "
                                               "keeps states and potentials, the reverse pass recomputes nothing"}
    return out


def batched_leg(torch, lenia, inputs, stream, steps=200):
    """256 single-channel localized-gene worlds of sides {64,128,256,512},
    R in 8..16, in one batch (CUDA graph per two steps) vs one plain
    1024^2 world of the same recipe, per site-step."""
    worlds = inputs.batched_worlds(live=True)
    sites = sum(w.sites for w in worlds)
    batch = lenia.lenia_batch_init(worlds, autotune=True, stream=stream)
    try:
        A = [torch.from_numpy(w.A).cuda() for w in worlds]
        P = [torch.from_numpy(w.P).cuda() for w in worlds]
        lenia.lenia_batch_rollout(batch, A, P, 4, stream)    # capture + warm-up
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        torch.cuda.nvtx.range_push("batched_timed")       # the timed launches, for ncu --nvtx-include
        lenia.lenia_batch_rollout(batch, A, P, steps, stream)
        torch.cuda.nvtx.range_pop()
        e1.record(stream)
        torch.cuda.synchronize()
        lenia.lenia_batch_check(batch)
        ms = e0.elapsed_time(e1)
        paths = [lenia.lenia_batch_conv_path(batch, i) for i in range(len(worlds))]
        shapes = {}
        for i, w in enumerate(worlds):
            if w.height not in shapes:
                kind, prm = lenia.lenia_batch_epilogue_shape(batch, i)
                shapes[w.height] = ({0: f"tiled, {prm} rows per thread",
                                     1: f"queued streaming, {prm} bands per world",
                                     2: f"tiled, 4 columns x {prm} rows per thread"}.get(kind, "own step"))
    finally:
        lenia.lenia_batch_destroy(batch)
    plain = inputs.localized_single_channel()
    cfg, ks = lenia.config_from_world(plain)
    ctx = lenia.lenia_init(cfg, ks, stream)
    try:
        a, p = torch.from_numpy(plain.A).cuda(), torch.from_numpy(plain.P).cuda()
        lenia.lenia_rollout(ctx, a, p, 4, None, stream)
        torch.cuda.synchronize()
        e0.record(stream)
        lenia.lenia_rollout(ctx, a, p, steps, None, stream)
        e1.record(stream)
        torch.cuda.synchronize()
        plain_ms = e0.elapsed_time(e1)
    finally:
        lenia.lenia_destroy(ctx)
    v = sites * steps / (ms / 1e3)
    pv = plain.sites * steps / (plain_ms / 1e3)
    return {"workload": f"{len(worlds)} worlds, sides 64-512, R 8..16, localized mu/sigma, {sites} sites",
            "steps": steps, "ms_per_step": ms / steps, "value": v, "unit": UNIT,
            "alg_bytes_per_site": 24, "frac_of_hbm": v * 24 / 1e9 / _peaks()[0],
            "fft_worlds": paths.count(lenia.CONV_FFT), "direct_worlds": paths.count(lenia.CONV_DIRECT),
            "epilogue_shape_by_side": {str(k): v for k, v in sorted(shapes.items())},
            "plain_1024_single_world": {"ms_per_step": plain_ms / steps, "value": pv},
            "batched_over_plain": v / pv}


def small_legs(torch, lenia, inputs, stream, fp32_peak=None):
    """The two small configurations as rollouts through lenia_rollout: the
    64^2 one-kernel world with global genes (100 steps; launch- and
    latency-bound, reported in us per step), on its automatic (FFT) route
    and on the direct route (one thread-block cluster), and the 1024^2 one-channel world
    with localized mu/sigma (1000 steps; reported against the HBM and FP32
    peaks; its state, ~12 MB, stays in L2)."""
    out = {}
    for name, w, steps, cp in (("c1", inputs.single_kernel_global(), 100, lenia.CONV_AUTO),
                               ("c1_direct_route", inputs.single_kernel_global(), 100, lenia.CONV_DIRECT),
                               ("c2", inputs.localized_single_channel(), 1000, lenia.CONV_AUTO)):
        cfg, ks = lenia.config_from_world(w, cp)
        ctx = lenia.lenia_init(cfg, ks, stream)
        try:
            a = torch.from_numpy(w.A).cuda()
            p = torch.from_numpy(w.P).cuda() if w.P is not None else None
            lenia.lenia_rollout(ctx, a, p, 10, None, stream)          # warm-up
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            lenia.lenia_rollout(ctx, a, p, steps, None, stream)
            e1.record(stream)
            torch.cuda.synchronize()
            lenia.lenia_check(ctx)
            ms = e0.elapsed_time(e1)
            path = lenia.lenia_conv_path(ctx)
            lps = lenia.lenia_launches_per_step(ctx)
            route = lenia.lenia_rollout_route(ctx)
        finally:
            lenia.lenia_destroy(ctx)
        v = w.sites * steps / (ms / 1e3)
        alg = 8 + (16 if w.P is not None else 0)          # A in/out, plus mu and sigma in/out
        r = {"workload": f"{w.height}x{w.width}, {w.n_channels} channel, {w.n_kernels} kernel R={w.kernels[0].radius}, "
                         + ("localized mu/sigma, gene maintenance" if w.P is not None else "global genes"),
             "steps": steps, "us_per_step": ms * 1e3 / steps, "value": v, "unit": UNIT,
             "conv_path": "fft" if path == lenia.CONV_FFT else "direct",
             "rollout": {lenia.ROUTE_STEPS: f"{lps} launches per step, pairs of steps replayed from a CUDA graph",
                         lenia.ROUTE_COOPERATIVE: "one cooperative launch",
                         lenia.ROUTE_CLUSTER: "one thread-block cluster"}.get(route, "?"),
             "launches_per_step": lps if route == lenia.ROUTE_STEPS else 1.0 / steps,
             "alg_bytes_per_site": alg, "frac_of_hbm": v * alg / 1e9 / _peaks()[0]}
        if fp32_peak and path == lenia.CONV_FFT:
            fl = fft_flops(w.height, w.width, w.n_channels, w.n_kernels)
            r["fp32_fft_frac_of_step"] = fl * steps / (ms / 1e3) / 1e12 / fp32_peak
        out[name] = r
    return out


def evolve_leg(torch, lenia, inputs, stream, plain_ms, steps=100):
    """The headline world with Algorithm 2's evolutionary lines switched on:
    an 8-column wall, one mutation and one penalisation per step (seeded
    events, r_oxy = 4, square half-size 16), against the plain step."""
    w = inputs.multi_channel(matched=True)
    H, W = w.height, w.width
    cfg, ks = lenia.config_from_world(w)
    ctx = lenia.lenia_init(cfg, ks, stream)
    try:
        lenia.lenia_set_walls(ctx, inputs.wall_strip(H, W, W // 2, 8))
        evs = [lenia.events_struct(inputs.evolution_events(w, s, gamma_mut=1.0, gamma_pen=0.2, mut_half=16,
                                                            r_oxy=4))
               for s in range(steps + 3)]
        bufs = [(torch.from_numpy(w.A).cuda(), torch.from_numpy(w.P).cuda())]
        bufs.append((torch.empty_like(bufs[0][0]), torch.empty_like(bufs[0][1])))
        st = torch.zeros((steps + 3, w.n_channels, 3), dtype=torch.float32, device="cuda")

        def step(i):
            (a, p), (a2, p2) = bufs[i % 2], bufs[(i + 1) % 2]
            lenia.lenia_step_evolve(ctx, a, p, a2, p2, evs[i], st[i], None, None, stream)

        for i in range(3):
            step(i)
        torch.cuda.synchronize()
        # timed without per-launch events, then a separate profiled region
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for i in range(steps):
            step(3 + i)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / steps
        n_prof = min(steps, 50)
        lenia.lenia_profile_start(ctx, 16 * n_prof)
        for i in range(n_prof):
            step(3 + i)
        torch.cuda.synchronize()
        prof = lenia.lenia_profile_stop(ctx)
        lenia.lenia_check(ctx)
    finally:
        lenia.lenia_destroy(ctx)
    sites = H * W
    disk_ms = prof["pen_disk"][0] / max(1, prof["pen_disk"][1]) if "pen_disk" in prof else 0.0
    # the disk pass reads the not-Delta_sum byte and the alpha byte of every
    # site and writes only the few gene values it changes
    disk_bytes = sites * 2
    return {"workload": "2048x2048, 3 channels, 15 kernels R=18, walls + mutation + penalisation each step",
            "steps": steps, "ms_per_step": ms, "value": sites / (ms / 1e3), "unit": UNIT,
            "over_plain_step": ms / plain_ms if plain_ms else None,
            "kernels_ms": {k: v[0] / max(1, v[1]) for k, v in prof.items()},
            "disk_pass_gbs": disk_bytes / (disk_ms / 1e3) / 1e9 if disk_ms > 0 else None,
            "stats_finite": bool(torch.isfinite(st).all())}


def rings_leg(torch, lenia, inputs, stream, steps=100):
    """The paper's own configuration (Section 2.1, 2.4): 512 x 1024 torus,
    3 channels, 15 two-bump kernels of radius 12 cut into 24 rings, all nine
    gene types localized per kernel and site (135 gene planes), maintenance
    on, potential alpha test."""
    w = inputs.ring_world()
    w.alpha_on = 1
    cfg, ks = lenia.config_from_world(w)
    ctx = lenia.lenia_init(cfg, ks, stream)
    try:
        bufs = [(torch.from_numpy(w.A).cuda(), torch.from_numpy(w.P).cuda())]
        bufs.append((torch.empty_like(bufs[0][0]), torch.empty_like(bufs[0][1])))
        st = torch.zeros((steps + 3, w.n_channels, 3), dtype=torch.float32, device="cuda")

        def step(i):
            (a, p), (a2, p2) = bufs[i % 2], bufs[(i + 1) % 2]
            lenia.lenia_step(ctx, a, p, a2, p2, st[i], stream)

        for i in range(3):
            step(i)
        torch.cuda.synchronize()
        # timed without per-launch events, then a separate profiled region
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for i in range(steps):
            step(3 + i)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / steps
        n_prof = min(steps, 50)
        lenia.lenia_profile_start(ctx, 8 * n_prof)
        for i in range(n_prof):
            step(3 + i)
        torch.cuda.synchronize()
        prof = lenia.lenia_profile_stop(ctx)
        lenia.lenia_check(ctx)
        path = lenia.lenia_conv_path(ctx)
    finally:
        lenia.lenia_destroy(ctx)
    sites = w.sites
    n_planes = w.n_planes * w.n_kernels
    alg = 3 * 4 * 2 + n_planes * 4 * 2
    epi = prof.get("epilogue", (0.0, 1))
    epi_ms = epi[0] / max(1, epi[1])
    return {"workload": "512x1024, 3 channels, 15 two-bump kernels R=12 in 24 rings, all 9 gene types localized "
                        f"({n_planes} gene planes)",
            "steps": steps, "ms_per_step": ms, "value": sites / (ms / 1e3), "unit": UNIT,
            "conv_path": "fft" if path == lenia.CONV_FFT else "direct",
            "ring_planes": w.n_channels * w.n_rings, "alg_bytes_per_site": alg,
            "epilogue_frac_of_hbm": (alg * sites / (epi_ms / 1e3) / 1e9) / _peaks()[0] if epi_ms > 0 else None,
            "kernels_ms": {k: v[0] / max(1, v[1]) for k, v in prof.items()},
            "real_time_goal_steps_per_s": 20, "steps_per_s": 1e3 / ms,
            "stats_finite": bool(torch.isfinite(st).all())}


def _kernel_taps(lenia, ctx, world):
    """Non-zero taps of each kernel and the Toeplitz K steps (16 input columns
    each) that the tensor-core route issues per kernel and 256 x 32 tile."""
    taps, ksteps = [], []
    Rm = max(k.radius for k in world.kernels)
    for k, kd in enumerate(world.kernels):
        Kw = lenia.lenia_kernel_weights(ctx, k, kd.radius)
        R = kd.radius
        taps.append(int((Kw != 0).sum()))
        n = 0
        for dy in range(-R, R + 1):
            nz = np.nonzero(Kw[dy + R])[0]
            if len(nz):
                dmin, dmax = int(nz[0]) - R, int(nz[-1]) - R
                n += (dmax + Rm + 31) // 16 - (dmin + Rm) // 16 + 1
        ksteps.append(n)
    return taps, ksteps


def _time_steps(torch, lenia, ctx, A, P, A2, P2, stream, n):
    for _ in range(3):
        lenia.lenia_step(ctx, A, P, A2, P2, None, stream)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(n):
        lenia.lenia_step(ctx, A, P, A2, P2, None, stream)
    e1.record(stream)
    torch.cuda.synchronize()
    step_ms = e0.elapsed_time(e1) / n
    lenia.lenia_profile_start(ctx, 8 * n)
    for _ in range(n):
        lenia.lenia_step(ctx, A, P, A2, P2, None, stream)
    torch.cuda.synchronize()
    prof = lenia.lenia_profile_stop(ctx)
    lenia.lenia_check(ctx)
    return step_ms, {k: v[0] / max(1, v[1]) for k, v in prof.items()}


def direct_leg(torch, lenia, inputs, stream, fp32_peak=None, bf16_peak=None, steps=50, only=None):
    """The direct convolution routes.  FP32 direct sums (TMA-staged tiles,
    kernels over grid z): the 64^2 one-kernel world (R = 13) as a rollout, and
    R = 5 worlds where the automatic choice is the direct path (1024^2 one
    channel; 2048^2 three channels, 15 kernels).  Tensor cores (BF16 Toeplitz
    products): the headline 2048^2 world (R = 18) with BF16 operands and with
    the high/low split, against its FFT route; tensor work is counted as
    issued (zero-padded band) and as useful (non-zero taps)."""
    out = {}
    w = inputs.single_kernel_global()
    cfg, ks = lenia.config_from_world(w, lenia.CONV_DIRECT)
    if only not in (None, "c1_direct"):
        cfg = None
    ctx = lenia.lenia_init(cfg, ks, stream) if cfg is not None else None
    try:
        if ctx is None:
            raise StopIteration
        a = torch.from_numpy(w.A).cuda()
        lenia.lenia_rollout(ctx, a, None, 10, None, stream)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        lenia.lenia_rollout(ctx, a, None, 100, None, stream)
        e1.record(stream)
        torch.cuda.synchronize()
        lenia.lenia_check(ctx)
        route = {lenia.ROUTE_STEPS: "launches per step (graph)", lenia.ROUTE_COOPERATIVE: "one cooperative launch",
                 lenia.ROUTE_CLUSTER: "one thread-block cluster"}.get(lenia.lenia_rollout_route(ctx), "?")
        out["c1_direct"] = {"workload": "64x64, 1 channel, 1 kernel R=13, global genes, 100-step rollout, direct path",
                            "us_per_step": e0.elapsed_time(e1) * 1e3 / 100, "route": route}
    except StopIteration:
        pass
    finally:
        if ctx is not None:
            lenia.lenia_destroy(ctx)
    cases = (("r5_1024", inputs.localized_single_channel(R=5), lenia.CONV_AUTO),
             ("r5_2048_c3", inputs.multi_channel(R=5, matched=True), lenia.CONV_AUTO),
             ("c3_fft", inputs.multi_channel(matched=True), lenia.CONV_FFT),
             ("c3_bf16", inputs.multi_channel(matched=True), lenia.CONV_DIRECT_BF16),
             ("c3_bf16x3", inputs.multi_channel(matched=True), lenia.CONV_DIRECT_BF16X3))
    for name, w, path in cases:
        if only is not None and name != only:
            continue
        cfg, ks = lenia.config_from_world(w, path)
        ctx = lenia.lenia_init(cfg, ks, stream)
        try:
            A, P = torch.from_numpy(w.A).cuda(), torch.from_numpy(w.P).cuda()
            A2, P2 = torch.empty_like(A), torch.empty_like(P)
            step_ms, kern = _time_steps(torch, lenia, ctx, A, P, A2, P2, stream, steps)
            used = lenia.lenia_conv_path(ctx)
            taps, ksteps = _kernel_taps(lenia, ctx, w)
        finally:
            lenia.lenia_destroy(ctx)
        conv_ms = sum(v for k, v in kern.items() if k in ("direct_conv", "rows_r2c", "cols_conv", "rows_c2r"))
        useful = 2.0 * sum(taps) * w.sites
        r = {"workload": f"{w.height}x{w.width}, {w.n_channels} channels, {w.n_kernels} kernels R={w.kernels[0].radius}",
             "conv_path": {1: "fft", 2: "direct_fp32", 3: "direct_bf16", 4: "direct_bf16x3"}[used],
             "ms_per_step": step_ms, "value": w.sites / (step_ms / 1e3), "unit": UNIT, "conv_ms": conv_ms,
             "kernels_ms": kern, "useful_conv_tflops": useful / (conv_ms / 1e3) / 1e12 if conv_ms else None}
        if used == lenia.CONV_DIRECT and fp32_peak:
            r["fp32_frac"] = r["useful_conv_tflops"] / fp32_peak
        if used in (lenia.CONV_DIRECT_BF16, lenia.CONV_DIRECT_BF16X3):
            terms = 1 if used == lenia.CONV_DIRECT_BF16 else 3
            issued = 2.0 * sum(ksteps) * 16 * 32 * 256 * terms * (w.sites / (32 * 256))
            r["issued_tensor_tflops"] = issued / (conv_ms / 1e3) / 1e12
            r["issued_over_useful"] = issued / useful
            if bf16_peak:
                r["tensor_frac_of_bf16_peak"] = r["issued_tensor_tflops"] / bf16_peak
        out[name] = r
    return out


def max_over_ranks(values, torch, device=None):
    """Element-wise max of a list of floats over all ranks (identity at N = 1)."""
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return [float(v) for v in values]
    t = torch.tensor(values, dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(v) for v in t]


def job_value(world_size, sites_per_rank, steps, slowest_ms):
    """Whole-job throughput of independent replicas: every rank's site-steps
    over the slowest rank's time."""
    return world_size * sites_per_rank * steps / (slowest_ms / 1e3)


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


class OracleSample:
    """The FP64 oracle as it stands, on this host's cores, over bounded random
    samples of the workload's sites (each site: 15 direct potentials, 30 gene
    diffusions, growth, alpha mask and update)."""

    def __init__(self):
        import oracle
        from paper_2304_05639_gb300 import inputs
        oracle.build()
        self.oracle, self.inputs = oracle, inputs
        self.world = inputs.multi_channel(matched=True)
        self.rng = inputs.Rng(99)
        self.rate = None

    def run(self, n: int):
        ys = self.rng.integers(n, 0, self.world.height - 1)
        xs = self.rng.integers(n, 0, self.world.width - 1)
        t0 = time.perf_counter()
        self.oracle.step_sites(self.world, ys, xs)
        return time.perf_counter() - t0

    def sites_for(self, seconds: float) -> int:
        if self.rate is None:
            self.rate = 1024 / max(self.run(1024), 1e-4)
        return int(min(2_000_000, max(256, self.rate * seconds)))

    def describe(self, n, dt):
        return {"value": n / dt, "unit": UNIT, "cores": self.oracle.num_threads(), "kind": "oracle",
                "sample": f"{n} random sites of the 2048^2 workload, one step each "
                          f"({dt:.2f} s; FP64 direct sums)"}


def cpu_baseline(seconds_target: float = 15.0):
    s = OracleSample()
    n = s.sites_for(seconds_target)
    return s.describe(n, s.run(n))


def run_reference(args):
    """The reference arm: the FP64 CPU oracle as it stands, each timed step a
    bounded random sample of the workload's sites (one step each).  value is
    sites per second over the timed samples; ms_per_step is the measured time
    of one sampled step, and the time a full 2048^2 step would take at that
    rate is given beside it, labelled as extrapolated."""
    ws, rank, _ = _dist()
    if rank != 0:
        return 0
    s = OracleSample()
    per_step = max(0.25, 120.0 / max(1, args.steps + args.warmup))
    n = s.sites_for(per_step)
    vals, tot = [], 0.0
    for i in range(args.warmup + args.steps):
        dt = s.run(n)
        if i >= args.warmup:
            vals.append(n / dt)
            tot += dt
    v = len(vals) * n / tot
    cb = s.describe(n * len(vals), tot)
    line = {"metric": METRIC, "value": v, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": tot / len(vals) * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "impl": "reference",
            "config": workload_config(ws), "conv_path": "direct FP64 sums (CPU oracle)",
            "sites_per_step": n,
            "step_sample": f"each timed step is {n} random sites of the 2048^2 workload (not the whole torus)",
            "ms_per_full_step_extrapolated": 2048 * 2048 / v * 1e3,
            "cpu_baseline": {**cb, "value": v},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "gpu_launches": 0}
    print(json.dumps(line), flush=True)
    return 0


def run_ours(args):
    import torch
    ws, rank, local = _dist()
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    else:
        torch.cuda.set_device(0)
    dev = torch.device("cuda", torch.cuda.current_device())

    from paper_2304_05639_gb300 import build, inputs, lenia
    if rank == 0 or ws == 1:
        build.build()
    if ws > 1:
        torch.distributed.barrier()
    if args.size == 2048:
        world = inputs.multi_channel(matched=True)
    else:   # same recipe on a smaller torus (profiling captures)
        world = inputs.multi_channel(H=args.size, W=args.size, patch=max(16, args.size // 8), matched=True)
    cfg, ks = lenia.config_from_world(world, args.conv_path)
    stream = torch.cuda.current_stream(dev)
    ctx = lenia.lenia_init(cfg, ks, stream)
    H, W = world.height, world.width
    sites = H * W
    A = torch.from_numpy(world.A).to(dev)
    P = torch.from_numpy(world.P).to(dev)
    A2, P2 = torch.empty_like(A), torch.empty_like(P)
    stats = torch.zeros((args.steps + args.warmup, world.n_channels, 3), dtype=torch.float32, device=dev)

    # every step advances the same live state (A, P) into (A2, P2): the
    # inputs (551 MB) are larger than L2, so no step reads them from cache
    def step(i):
        lenia.lenia_step(ctx, A, P, A2, P2, stats[i], stream)

    for i in range(args.warmup):
        step(i)
    torch.cuda.synchronize()
    launches_per_step = lenia.lenia_launches_per_step(ctx)
    # sites whose genes survive the step (alpha = 1)
    alpha1 = int((P2 != 0).all(dim=0).all(dim=0).sum()) if P2.numel() else 0
    # FP32 FMA throughput of this GPU, measured (the denominator of the FFT
    # passes' FP32 fraction), before the timed region
    fp32_scalar, fp32_pair = lenia.lenia_measure_fp32_peak(stream)

    # the timed region: plain steps, no per-launch events
    clocks = Clocks(torch.cuda.current_device()) if rank == 0 else None
    if ws > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for i in range(args.steps):
        step(args.warmup + i)
    e1.record(stream)
    torch.cuda.synchronize()
    if ws > 1:
        torch.distributed.barrier()
    ms = e0.elapsed_time(e1)
    clk = clocks.stop() if clocks else None

    # a second, separate region times each launch (CUDA events around every
    # launch on the launching stream) for the per-kernel figures
    prof_steps = min(args.steps, 200)
    lenia.lenia_profile_start(ctx, launches_per_step * prof_steps + 8)
    for i in range(prof_steps):
        step(i)
    torch.cuda.synchronize()
    prof = lenia.lenia_profile_stop(ctx)

    # end to end through the public host-buffer entry points: a serving loop of
    # independent host worlds (pinned buffers), each step uploading its
    # world's A and P and downloading A', P' and the stats; the uploads of one
    # step overlap the downloads of the previous one
    pin = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory()
    hA, hP = pin(world.A), pin(world.P)
    outs = [(torch.empty_like(hA).pin_memory(), torch.empty_like(hP).pin_memory(),
             torch.zeros((world.n_channels, 3), dtype=torch.float32).pin_memory()) for _ in range(2)]
    hst = outs[0][2]
    e2e_steps = max(4, min(args.steps, 20))
    e2e_s = float("nan")
    e2e_rounds = []
    if not args.no_e2e:
        lenia.lenia_step_host(ctx, hA, hP, outs[0][0], outs[0][1], outs[0][2], stream)
        torch.cuda.synchronize()
        # three rounds of e2e_steps steps; the median round is reported (the
        # host link is shared, and one slow round should not set the number)
        for _ in range(3):
            t0 = time.perf_counter()
            for i in range(e2e_steps):
                oA, oP, ost = outs[i % 2]
                lenia.lenia_step_host_async(ctx, hA, hP, oA, oP, ost, stream)
            lenia.lenia_host_wait(ctx, stream)
            e2e_rounds.append(time.perf_counter() - t0)
        e2e_s = sorted(e2e_rounds)[1]

    t_max, e2e_max = max_over_ranks([ms, e2e_s if e2e_s == e2e_s else 0.0], torch, dev)
    if e2e_s != e2e_s:
        e2e_max = float("nan")

    ok_stats = bool(torch.isfinite(stats).all())
    path = lenia.lenia_conv_path(ctx)
    fft_ref = None
    if ws == 1 and not args.no_extras and path == lenia.CONV_FFT:
        fft_ms = sum(prof[k][0] / max(1, prof[k][1]) for k in ("rows_r2c", "cols_conv", "rows_c2r") if k in prof)
        fft_ref = cufft_yardstick(torch, lenia, ctx, world, stream, fft_ms)
    lenia.lenia_destroy(ctx)
    if rank != 0:
        if ws > 1:
            torch.distributed.destroy_process_group()
        return 0

    value = job_value(ws, sites, args.steps, t_max)
    hbm, peak_kind = _peaks()
    # dominant kernel: the largest share of the timed region
    dom = max(prof.items(), key=lambda kv: kv[1][0]) if prof else ("none", (0.0, 1))
    dom_ms = dom[1][0] / max(1, dom[1][1])
    # the epilogue moves all of the method's bytes (A and P in and out); the
    # FFT passes move only implementation intermediates
    alg_bytes = ALG_BYTES_PER_SITE * sites if dom[0] == "epilogue" else 0
    achieved = alg_bytes / (dom_ms / 1e3) / 1e9 if dom_ms > 0 else 0.0
    traffic = _traffic(dom[0]) if args.size == 2048 else None
    step_traffic = (_traffic("step", "step_traffic.json", "dram_bytes_per_step")
                    if args.size == 2048 and path == lenia.CONV_FFT else None)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t_max / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": workload_config(ws, args.size), "conv_path": "fft" if path == lenia.CONV_FFT else "direct",
        "roofline": {"bound": "hbm", "kernel": dom[0], "achieved": achieved, "peak": hbm,
                     "peak_kind": peak_kind, "unit": "GB/s", "frac": achieved / hbm,
                     "traffic": traffic,
                     "traffic_gbs": (traffic / (dom_ms / 1e3) / 1e9) if traffic else None,
                     "alg_bytes_per_site": ALG_BYTES_PER_SITE,
                     "step_frac": (ALG_BYTES_PER_SITE * sites * args.steps / (t_max / 1e3) / 1e9) / hbm,
                     "step_traffic": step_traffic,
                     "step_dram_frac": (step_traffic * args.steps / (t_max / 1e3) / 1e9) / hbm
                     if step_traffic else None},
        "fp32": fp32_line(prof, H, W, fp32_scalar, fp32_pair),
        "kernels_ms": {k: {"avg_ms": v[0] / max(1, v[1]), "launches": v[1],
                           "share": v[0] / max(1e-9, sum(x[0] for x in prof.values()))}
                       for k, v in prof.items()},
        "e2e": {"value": job_value(ws, sites, e2e_steps, e2e_max * 1e3) if e2e_max == e2e_max else None,
                "unit": UNIT,
                "h2d_bytes_per_step": int(world.A.nbytes + world.P.nbytes),
                "d2h_bytes_per_step": int(world.A.nbytes + world.P.nbytes + hst.numel() * 4),
                "mode": "independent host worlds, lenia_step_host_async + lenia_host_wait, pinned buffers",
                "rounds_ms_per_step": [r * 1e3 / e2e_steps for r in e2e_rounds],
                "reported": "median of the rounds"},
        "gpu_launches": launches_per_step * args.steps,
        "clocks": clk,
        "stats_finite": ok_stats,
        "alpha1_sites": alpha1,
        "kernel_profile": f"per-launch CUDA events over {prof_steps} steps after the timed region",
    }
    if fft_ref is not None:
        line["fft_yardstick"] = fft_ref
    if not args.no_extras and ws == 1 and args.size == 2048:
        line["adjoint"] = adjoint_leg(torch, lenia, inputs, stream)
        line["batched"] = batched_leg(torch, lenia, inputs, stream)
        line["evolve"] = evolve_leg(torch, lenia, inputs, stream, t_max / args.steps)
        line["rings"] = rings_leg(torch, lenia, inputs, stream)
        line["small"] = small_legs(torch, lenia, inputs, stream, max(fp32_scalar, fp32_pair))
        line["direct"] = direct_leg(torch, lenia, inputs, stream, max(fp32_scalar, fp32_pair), _bf16_peak())
    if not args.no_cpu_baseline and ws == 1:
        line["cpu_baseline"] = cpu_baseline()
    print(json.dumps(line), flush=True)
    if ws > 1:
        torch.distributed.destroy_process_group()
    return 0


def spawn_ranks(argv, gpus):
    """--gpus N > 1 outside a torchrun environment: start N ranks of this
    script with torch.distributed.run on 127.0.0.1 and return their exit
    status (None when nothing needs spawning)."""
    if gpus <= 1 or "WORLD_SIZE" in os.environ:
        return None
    import socket
    sk = socket.socket()
    sk.bind(("127.0.0.1", 0))
    port = sk.getsockname()[1]
    sk.close()
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", f"--nproc-per-node={gpus}",
           "--master-addr=127.0.0.1", f"--master-port={port}", os.path.abspath(__file__)] + list(argv)
    return subprocess.call(cmd)


def run_rank_check(args):
    """CPU check of the rank plumbing (gloo, no GPU): every rank reports a
    made-up time (10 + rank ms), rank 0 prints the max over ranks, the world
    size and the job value the GPU path would compute from them."""
    import torch
    import torch.distributed as dist
    ws, rank, _ = _dist()
    if ws > 1:
        dist.init_process_group("gloo")
    t_max = max_over_ranks([10.0 + rank], torch)[0]
    if rank == 0:
        print(json.dumps({"n_gpus": ws, "ms_max": t_max, "value": job_value(ws, 1000, 1, t_max)}), flush=True)
    if ws > 1:
        dist.barrier()
        dist.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--rank-check", action="store_true",
                    help="check the multi-rank plumbing on CPU (gloo) and exit")
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true", help="skip the host-buffer end-to-end leg")
    ap.add_argument("--no-extras", action="store_true", help="skip the adjoint, batched-world, evolution, ring and small-world legs")
    ap.add_argument("--size", type=int, default=2048, help="torus side (2048 = the benchmark workload)")
    ap.add_argument("--conv-path", type=int, default=0, help="0 auto, 1 fft, 2 direct")
    ap.add_argument("--direct-case", default=None,
                    choices=["c1_direct", "r5_1024", "r5_2048_c3", "c3_fft", "c3_bf16", "c3_bf16x3"],
                    help="with --leg direct: run this case alone (for profiling)")
    ap.add_argument("--leg", default=None, choices=["adjoint", "batched", "evolve", "rings", "small", "direct"],
                    help="run only this extra leg (N = 1) and print its JSON object (for profiling)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    rc = spawn_ranks(sys.argv[1:], args.gpus)
    if rc is not None:
        return rc
    if args.rank_check:
        return run_rank_check(args)
    if args.impl == "reference":
        return run_reference(args)
    if args.leg:
        return run_leg(args)
    return run_ours(args)


def run_leg(args):
    import torch
    from paper_2304_05639_gb300 import build, inputs, lenia
    torch.cuda.set_device(0)
    build.build()
    stream = torch.cuda.current_stream()
    if args.leg == "adjoint":
        out = adjoint_leg(torch, lenia, inputs, stream)
    elif args.leg == "batched":
        out = batched_leg(torch, lenia, inputs, stream, steps=args.steps)
    elif args.leg == "evolve":
        out = evolve_leg(torch, lenia, inputs, stream, None, steps=args.steps)
    elif args.leg == "small":
        out = small_legs(torch, lenia, inputs, stream, max(lenia.lenia_measure_fp32_peak(stream)))
    elif args.leg == "direct":
        out = direct_leg(torch, lenia, inputs, stream, max(lenia.lenia_measure_fp32_peak(stream)), _bf16_peak(),
                         steps=args.steps, only=args.direct_case)
    else:
        out = rings_leg(torch, lenia, inputs, stream, steps=args.steps)
    print(json.dumps({"leg": args.leg, **out}), flush=True)
    return 0


if __name__ == "__main__":
    sys.exit(main())
