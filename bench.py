#!/usr/bin/env python
"""Benchmark of the Chemora FP64 hot path on GB300: grid-point updates/s of
RK4 steps of the BSSN Einstein equations on a 128^3 periodic grid (24
evolved variables, 4th-order FD with mixed second derivatives, KO eps = 0.1,
1+log slicing, Gamma-driver shift, 3 ghost zones; flat space + uniform noise
of amplitude 1e-10, dt = h/4).

One step = one RK4 step (4 fused stage kernels + 4 ghost fills) of the whole
grid.  The state (462 MB) and the RK4 scratch (1.39 GB) exceed the 129 MB L2,
so no L2 flush is needed between steps.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl chemora|reference]

Under torchrun each rank advances its own replica (the path is a single grid
per GPU; no data-path collective) and rank 0 prints one JSON line.  The
reference arm times the FP64 CPU oracle on this host's cores.
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "FP64 grid-point updates/s (RK4 step, BSSN 128^3)"
UNIT = "grid-point updates/s"
N_DEFAULT = 128
GHOSTS = 3
NVARS = 24
SEED = 2


def _dist():
    from paper_1410_1764_gb300 import dist
    return dist.world()


class ClockSampler:
    """nvidia-smi SM clock and throttle-reason samples during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.Q,
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.t.join(timeout=2)
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def _workload(n):
    from paper_1410_1764_gb300 import synth
    st, h = synth.bssn_noise(n, n, n, GHOSTS, seed=SEED)
    return st, h


def _config(n, ws):
    return {"workload": "bssn_%d^3_flat_noise_1e-10" % n, "grid": [n, n, n], "nvars": NVARS,
            "ghosts": GHOSTS, "dt": "h/4", "fd_order": 4, "ko_eps": 0.1,
            "gauge": "1+log, Gamma-driver (eta=2)",
            "l2": "inputs larger than L2 (state %.0f MB + RK4 scratch %.0f MB)" % (
                NVARS * (n + 2 * GHOSTS) ** 3 * 8 / 1e6, 3 * NVARS * (n + 2 * GHOSTS) ** 3 * 8 / 1e6),
            "parallelism": "replicas x%d (one grid per GPU)" % ws}


# Frozen algorithmic flop count F of one BSSN right-hand side per point: the
# generator's count (add/sub/mul 1, fma 2, exp and reciprocal 1 each) on the
# CSE'd DAG of the direct (canonical) body of the phi-form equations, frozen
# so that no later change of the emitted bodies moves the roofline's
# numerator.  The fused RK update adds 13 flops per variable per RK4 step
# (3.25 per stage on average).
FROZEN_RHS_FLOPS_BSSN = 3760
RK_UPDATE_FLOPS = 3.25


def _profile_traffic(kernel_key):
    """DRAM traffic per launch of the timed stage kernel from the committed
    machine-readable ncu figures (profiles/bssn_stage_kernel_128.json), or
    None when they were taken on a different build of the kernel."""
    path = os.path.join(ROOT, "profiles", "bssn_stage_kernel_128.json")
    try:
        with open(path) as f:
            vals = json.load(f)
    except (OSError, ValueError):
        return None
    if vals.get("kernel_source_hash") != kernel_key:
        return None
    v = vals.get("dram_bytes_per_launch")
    return float(v) if isinstance(v, (int, float)) else None


def kernel_source_hash():
    """Hash of the code (comments and blank lines removed) of the sources the
    timed, run-time specialised BSSN stage kernel is built from: the device
    headers NVRTC compiles (of the generated bodies, the x/y-sharing one the
    profiled launch shape instantiates) and the part of the specialiser that
    writes the kernel source and the compiler options."""
    import hashlib
    import re
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_1410_1764_gb300", "csrc")
    for rel in ("bssn_kernels.cuh", "jit.cu", "stage.cuh", "device_types.cuh",
                "generated/gen_constants.cuh", "generated/gen_bssn_xy.cuh"):
        with open(os.path.join(csrc, rel)) as f:
            text = re.sub(r"/\*.*?\*/", "", f.read(), flags=re.S)
        if rel == "jit.cu":  # only what shapes the kernel: its source text and the options
            m = re.search(r"std::string kernel_source\(.*?\n}\n", text, flags=re.S)
            opts = [ln for ln in text.splitlines() if "opts = {" in ln or "opts.push_back" in ln]
            text = (m.group(0) if m else text) + "\n".join(opts)
        code = [ln.split("//", 1)[0].rstrip() for ln in text.splitlines()]
        h.update("\n".join(ln for ln in code if ln).encode())
    return h.hexdigest()[:16]


def _kernel_name(api, fp64_instr, variant, specialised):
    """The BSSN stage kernel the chosen launch shape runs: the direct body,
    the x lane-sharing body or the x lane + y shared-memory body (the last
    carries the prologue in its count); run-time specialised kernels are all
    named chemora_jit_stage."""
    if fp64_instr == api.opcount(api.BSSN)[0]:
        name, body = "bssn_stage_kernel", "direct"
    elif api.variant_info(api.BSSN, variant)[3] == 2:
        name, body = "bssn_xystage_kernel", "x/y-sharing"
    else:
        name, body = "bssn_xstage_kernel", "x-sharing"
    return "chemora_jit_stage (%s body)" % body if specialised else name


def cpu_baseline(n, nsteps=2, nz1=16):
    """The oracle, as it stands, on this host's cores: nsteps RK4 steps of the
    full grid; and on one core, one RK4 step of an n x n x nz1 periodic slab
    of the same recipe (same planes, fewer of them, to bound the time)."""
    import oracle
    oracle.lib()  # load (and, if stale, build) the library before the timed call
    st, h = _workload(n)
    t0 = time.perf_counter()
    oracle.rk4(oracle.BSSN, st, GHOSTS, h, 0.25 * h, nsteps)
    dt = time.perf_counter() - t0
    pts = n ** 3
    cores = oracle.num_threads()
    from paper_1410_1764_gb300 import synth
    st1, h1 = synth.bssn_noise(n, n, nz1, GHOSTS, seed=SEED)
    oracle.set_num_threads(1)
    try:
        t0 = time.perf_counter()
        oracle.rk4(oracle.BSSN, st1, GHOSTS, h1, 0.25 * h1, 1)
        dt1 = time.perf_counter() - t0
    finally:
        oracle.set_num_threads(cores)
    return {"value": pts * nsteps / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": "%d RK4 steps of the full %d^3 grid (%.1f s)" % (nsteps, n, dt),
            "value_1core": n * n * nz1 / dt1,
            "sample_1core": "1 RK4 step of a %d x %d x %d periodic slab, 1 thread (%.1f s)" % (n, n, nz1, dt1)}


# RK update FP64 instructions per variable per stage, averaged over the four
# stages: BSSN's classic rounding (2, 3, 3, 3) and the scalar-wave systems'
# contracted update (1, 2, 2, 2)
RK_FMA = 2.75
RK_FMA_WAVE = 1.75
ISSUE_PEAK = [None]  # FP64 instructions per second: SMs x 2 per clock x max clock


def _issue_frac(instr_per_point_stage, points_per_s):
    """FP64 issue fraction of a measured RK4 throughput (4 stages per step,
    every FP64 instruction an fma) against ISSUE_PEAK."""
    if not ISSUE_PEAK[0]:
        return None
    return instr_per_point_stage * 4 * points_per_s / ISSUE_PEAK[0]


def bench_patches(api, nsteps, npatch=64, seed=3, reps=5):
    """Batched BSSN patches (64 patches, sides U[16,96], g = 3, h = 1/64,
    flat + 1e-10 noise): updates/s of the batched schedule (one persistent
    launch per stage, graph-captured step) and of per-patch launches, each
    timed over nsteps RK4 steps, `reps` times with the two schedules
    alternating; the median and the min/max of the repeats are reported.
    With several ranks the patches are sharded (independent problems, no
    collective); each time is the maximum over ranks."""
    import torch
    from paper_1410_1764_gb300 import dist as D
    from paper_1410_1764_gb300 import synth
    states, dims, h = synth.bssn_patches(seed=seed, npatch=npatch)
    ws, rank, _ = D.world()
    mine = D.shard_patches(dims, ws)[rank]
    pts = int(sum(int(a) * int(b) * int(c) for a, b, c in dims))
    out = {"workload": "bssn_patches_%d_sides_16-96" % npatch, "interior_points": pts,
           "steps": nsteps, "repeats": reps, "ranks": ws}
    dt = 0.25 * h
    batches = {}
    for mode in (0, 1):
        b = api.Batch([tuple(int(v) for v in dims[p]) for p in mine], GHOSTS, h, kind=api.BSSN)
        for q, p in enumerate(mine):
            b.state(q).copy_(torch.from_numpy(states[p]))
        b.step(dt, 1, mode=mode)  # warm-up (captures the batched step's graph)
        batches[mode] = b
    torch.cuda.synchronize()
    clocks = ClockSampler(torch.cuda.current_device())
    clocks.start()
    ms = {0: [], 1: []}
    for _ in range(reps):
        for mode in (0, 1):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record()
            batches[mode].step(dt, nsteps, mode=mode)
            e1.record()
            torch.cuda.synchronize()
            ms[mode].append(D.max_over_ranks(e0.elapsed_time(e1), device="cuda"))
    out["clocks"] = clocks.stop()
    del batches
    for mode, key in ((0, "batched"), (1, "per_patch")):
        ups = sorted(pts * nsteps / (t * 1e-3) for t in ms[mode])
        out[key] = statistics.median(ups)
        out[key + "_min"], out[key + "_max"] = ups[0], ups[-1]
    out["speedup"] = out["batched"] / out["per_patch"]
    pair = sorted(b / a for a, b in zip(ms[0], ms[1]))  # per repeat: per-patch time / batched time
    out["speedup_min"], out["speedup_max"] = pair[0], pair[-1]
    instr = api.opcount(api.BSSN)[0] + NVARS * RK_FMA  # direct body: both schedules
    out["fp64_instr_per_point_per_stage"] = instr
    out["fp64_issue_frac"] = {k: _issue_frac(instr, out[k] / max(1, ws)) for k in ("batched", "per_patch")}
    return out


def bench_adjoint(api, reps=3):
    """Variable-speed wave 128^3, 50 RK4 steps, 512 receivers, checkpoint
    every 10 steps: time of the forward pass alone (chemora_rk4_step) and of
    chemora_adjoint_rk4 (forward with checkpoints + reverse sweep with
    segment recomputation), CUDA events on the current stream, `reps`
    alternating repeats (median, min, max); ratio = (adjoint - forward) /
    forward of the medians."""
    import torch
    from paper_1410_1764_gb300 import synth
    n, g, nsteps, ck = 128, 2, 50, 10
    y0, c, recv, h, seed_true = synth.adjoint_problem(n=n, g=g)
    dt = 0.25 * h
    sysm = api.make_system(api.WAVE_VARC, n, n, n, h)
    C = torch.from_numpy(c).cuda()
    Y0 = torch.from_numpy(y0).cuda()
    sysm.set_speed(C)
    data = [0.0] * len(recv)
    # warm up both paths
    y = Y0.clone()
    sysm.rk4_step(y, dt, 2)
    api.adjoint_rk4(sysm, Y0, C, dt, 2, ck, recv, data)
    torch.cuda.synchronize()
    clocks = ClockSampler(torch.cuda.current_device())
    clocks.start()
    tf, ta = [], []
    for _ in range(reps):
        y = Y0.clone()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e2 = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record()
        sysm.rk4_step(y, dt, nsteps)
        e1.record()
        api.adjoint_rk4(sysm, Y0, C, dt, nsteps, ck, recv, data)  # synchronises its stream at the end
        e2.record()
        torch.cuda.synchronize()
        tf.append(e0.elapsed_time(e1))
        ta.append(e1.elapsed_time(e2))
    clk = clocks.stop()
    f, a = statistics.median(tf), statistics.median(ta)
    return {"workload": "varc_wave_128^3_50_steps_512_receivers_ckpt10", "forward_ms": f,
            "adjoint_total_ms": a, "backward_over_forward": (a - f) / f, "repeats": reps,
            "forward_ms_min_max": [min(tf), max(tf)], "adjoint_ms_min_max": [min(ta), max(ta)],
            "clocks": clk}


def bench_wave(api, cases=("32", "256")):
    """The two scalar-wave workloads at their configured lengths: 32^3 plane
    wave (100 RK4 steps) and 256^3 Gaussian pulses (200 steps), dt = h/4,
    after autotuning (graph-replayed steps or, where the autotuner finds it
    faster, launch-chained stages); SM clocks sampled per workload."""
    import torch
    from paper_1410_1764_gb300 import synth
    out = {}
    for name, n, steps, make in (("wave_32^3_plane", 32, 100, lambda: synth.plane_wave(32, 2)),
                                 ("wave_256^3_pulses", 256, 200, lambda: synth.gaussian_pulses(256, 2, seed=1))):
        if str(n) not in cases:
            continue
        y0, h = make()
        sysm = api.make_system(api.WAVE, n, n, n, h)
        t = torch.from_numpy(y0).cuda()
        v, shape, _ = sysm.autotune(t)
        sysm.rk4_step(t, 0.25 * h, 3)
        torch.cuda.synchronize()
        clocks = ClockSampler(torch.cuda.current_device())
        clocks.start()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        sysm.rk4_step(t, 0.25 * h, steps)
        e1.record()
        torch.cuda.synchronize()
        clk = clocks.stop()
        ms = e0.elapsed_time(e1)
        ups = n ** 3 * steps / (ms * 1e-3)
        instr = sysm.opcount()[0] + 2 * RK_FMA_WAVE
        out[name] = {"updates_per_s": ups, "ms_per_step": ms / steps, "steps": steps, "clocks": clk,
                     "block": list(shape),
                     "launch_chained": sysm.set_chain(-1),
                     "sharing": api.variant_info(api.WAVE, v)[3],
                     "fp64_instr_per_point_per_stage": instr, "fp64_issue_frac": _issue_frac(instr, ups)}
    return out


def bench_orders(api, n=128, steps=10):
    """Scalar-wave systems at every compiled finite-difference order on n^3
    (Gaussian pulses; the first-order form starts with v = grad u = 0):
    updates/s and FP64 instructions per point of the order-p body."""
    import json as _json
    import torch
    from paper_1410_1764_gb300 import synth
    counts = _json.load(open(os.path.join(ROOT, "paper_1410_1764_gb300", "csrc", "generated",
                                          "opcounts.json")))
    out = {}
    for kind, name in ((api.WAVE, "wave"), (api.WAVE1, "wave1")):
        for order in (2, 4, 6, 8):
            g = max(2, order // 2)
            y0, h = synth.gaussian_pulses(n, g, seed=1)
            if kind == api.WAVE1:
                y0 = np.concatenate([y0, np.zeros((3,) + y0.shape[1:])])
            sysm = api.make_system(kind, n, n, n, h, params=api.default_params(fd_order=order), nghost=g)
            t = torch.from_numpy(np.ascontiguousarray(y0)).cuda()
            sysm.autotune(t)
            sysm.rk4_step(t, 0.25 * h, 2)
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            sysm.rk4_step(t, 0.25 * h, steps)
            e1.record()
            torch.cuda.synchronize()
            key = ("wave_o%d" % order) if (kind == api.WAVE and order != 4) else (
                "wave" if kind == api.WAVE else "wave1_o%d" % order)
            ups = n ** 3 * steps / (e0.elapsed_time(e1) * 1e-3)
            # the order-4 two-variable wave may run the x-lane / z-queue body
            rhs_instr = sysm.opcount()[0] if key == "wave" else counts[key]["fp64_instructions"]
            instr = rhs_instr + (2 if kind == api.WAVE else 5) * RK_FMA_WAVE
            out["%s_o%d_%d^3" % (name, order, n)] = {
                "updates_per_s": ups, "fp64_instr_per_point_rhs": rhs_instr,
                "fp64_issue_frac": _issue_frac(instr, ups)}
    return out


def bench_amr(api, nc=128, steps=4):
    """Two-level refinement of the scalar wave: coarse 128^3 (h = 1/128) with
    the box [32, 96)^3 refined by 2 (fine 128^3 interior, 8-point buffer),
    Gaussian pulses on both levels, dt = h/4.  Updates counted per coarse
    step: coarse points + 2 x fine points (two fine substeps)."""
    import torch
    from paper_1410_1764_gb300 import synth
    lo, hi = (32, 32, 32), (96, 96, 96)
    H = 1.0 / nc
    amr = api.Amr(nc, lo, hi, H)
    yc, _ = synth.gaussian_pulses(nc, 2, seed=1)
    amr.state(0).copy_(torch.from_numpy(yc))
    nf = 2 * (hi[0] - lo[0])
    fine = amr.state(1)
    fine.zero_()
    # fine interior from the same pulses sampled at the fine points (x = lo H + f H/2)
    yf, _ = synth.gaussian_pulses(2 * nc, 8, seed=1)  # same recipe on the doubled grid
    off = 2 * lo[0]
    fine[:, 8:8 + nf, 8:8 + nf, 8:8 + nf].copy_(
        torch.from_numpy(np.ascontiguousarray(yf[:, 8 + off:8 + off + nf, 8 + off:8 + off + nf,
                                                  8 + off:8 + off + nf])))
    dt = 0.25 * H
    amr.step(dt, 1)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    amr.step(dt, steps)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / steps
    pts = nc ** 3 + 2 * nf ** 3
    return {"workload": "wave_amr_coarse128_fine_box_32-96", "ms_per_coarse_step": ms,
            "updates_per_s": pts / (ms * 1e-3), "coarse_points": nc ** 3, "fine_points": nf ** 3}


def bench_amr_bssn(api, nc=128, steps=2, reps=3, seed=5):
    """Two-level BSSN: coarse 128^3 (h = 1/128) with 8 refined boxes (one
    per octant, sides U[16,40] coarse points, buffer 12), flat space + 1e-10
    noise on both levels, coarse dt = h/4.  Updates per coarse step: coarse
    points + 2 x fine interior points.  The coarse stage kernel's launch
    shape is autotuned once (shared by both schedules).  Batched boxes (one
    persistent launch per fine RK stage over every box) against box-by-box
    launches, each timed over `steps` coarse steps, `reps` times
    alternating; medians."""
    import torch
    from paper_1410_1764_gb300 import synth
    boxes = synth.amr_boxes(seed, nc, lo=16, hi=40)
    H = 1.0 / nc
    r = synth.rng(seed + 1)
    ncf = [int(np.prod([2 * (hi[d] - lo[d]) for d in range(3)])) for lo, hi in boxes]
    pts = nc ** 3 + 2 * sum(ncf)
    amrs = {}
    for mode in (0, 1):
        a = api.AmrBoxes(api.BSSN, (nc, nc, nc), boxes, H)
        st, _ = synth.bssn_noise(nc, nc, nc, 3, None, r=synth.rng(seed + 2))
        a.state(0).copy_(torch.from_numpy(st))
        for b, (lo, hi) in enumerate(boxes):
            nf = [2 * (hi[d] - lo[d]) for d in range(3)]
            fb, _ = synth.bssn_noise(nf[0], nf[1], nf[2], 12, None, r=r)
            a.state(1 + b).copy_(torch.from_numpy(fb))
        variant = a.autotune()
        a.step(0.25 * H, 1, mode=mode)
        amrs[mode] = a
    torch.cuda.synchronize()
    ms = {0: [], 1: []}
    for _ in range(reps):
        for mode in (0, 1):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            amrs[mode].step(0.25 * H, steps, mode=mode)
            e1.record()
            torch.cuda.synchronize()
            ms[mode].append(e0.elapsed_time(e1) / steps)
    del amrs
    out = {"workload": "bssn_amr_coarse%d_8_boxes_sides_16-40" % nc, "coarse_points": nc ** 3,
           "coarse_variant": variant,
           "fine_points": sum(ncf), "boxes": [list(map(list, b)) for b in boxes], "coarse_steps": steps,
           "repeats": reps}
    for mode, key in ((0, "batched"), (1, "per_box")):
        m = statistics.median(ms[mode])
        out[key + "_ms_per_coarse_step"] = m
        out[key] = pts / (m * 1e-3)
    out["speedup"] = out["batched"] / out["per_box"]
    return out


def parity_check(sysm, state, h):
    """One right-hand side of the timed system (the run-time specialised
    kernel) on the state left by the timed steps, against the oracle's on
    the same input: the gate's per-variable scaled error max |a-b| /
    max(|b|, S_v) (S_v = max |b_v|; gate 1e-12) and, beside it, the raw
    pointwise relative error where |b| > 1e-3 S_v."""
    import oracle
    import torch
    oracle.lib()
    sysm.fill_ghosts(state)
    st = state.detach().cpu().numpy()
    a = sysm.rhs(state).detach().cpu().numpy()
    b = oracle.bssn_rhs(st, GHOSTS, h)
    g = GHOSTS
    a = a[:, g:-g, g:-g, g:-g].reshape(a.shape[0], -1)
    b = b[:, g:-g, g:-g, g:-g].reshape(b.shape[0], -1)
    S = np.abs(b).max(axis=1, keepdims=True)
    den = np.maximum(np.abs(b), np.where(S == 0, 1.0, S))
    err = np.abs(a - b)
    big = np.abs(b) > 1e-3 * S
    torch.cuda.synchronize()
    return {"what": "one RHS of the timed kernel vs the oracle on the post-benchmark state",
            "scaled_err": float((err / den).max()), "gate": 1e-12,
            "raw_rel_err_where_b_gt_1e-3_S": float((err[big] / np.abs(b[big])).max()) if big.any() else None}


def bench_constraints(api, sysm, state, n, reps=10):
    """BSSN constraints (Hamiltonian, momentum, Gamma-tilde constraint, 7
    outputs per point) on the timed 128^3 state: one launch of the direct
    generated body per call, ghosts filled first; CUDA events around `reps`
    launches on the current stream."""
    import json as _json
    import torch
    counts = _json.load(open(os.path.join(ROOT, "paper_1410_1764_gb300", "csrc", "generated",
                                          "opcounts.json")))["bssn_constraints"]
    out = torch.empty((7,) + tuple(state.shape[1:]), dtype=torch.float64, device=state.device)
    sysm.fill_ghosts(state)
    for _ in range(2):
        sysm.constraints(state, out)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        sysm.constraints(state, out)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / reps
    pps = n ** 3 / (ms * 1e-3)
    instr = counts["fp64_instructions"]
    return {"workload": "bssn_constraints_%d^3" % n, "ms_per_launch": ms, "points_per_s": pps,
            "fp64_instr_per_point": instr,
            "fp64_issue_frac": instr * pps / ISSUE_PEAK[0] if ISSUE_PEAK[0] else None}


def run_reference(args):
    ws, rank, _ = _dist()
    if rank != 0:
        return 0
    import oracle
    oracle.lib()  # load (and, if stale, build) the library before the timed steps
    n = args.n
    st, h = _workload(n)
    dt = 0.25 * h
    y = st
    for _ in range(args.warmup):
        y = oracle.rk4(oracle.BSSN, y, GHOSTS, h, dt, 1)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        y = oracle.rk4(oracle.BSSN, y, GHOSTS, h, dt, 1)
    el = time.perf_counter() - t0
    v = n ** 3 * args.steps / el
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": el / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": _config(n, 1),
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": oracle.num_threads(), "kind": "oracle",
                             "sample": "%d timed RK4 steps of the full %d^3 grid" % (args.steps, n)},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def run_chemora(args):
    import torch

    ws, rank, local = _dist()
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    from paper_1410_1764_gb300 import api

    n = args.n
    st_np, h = _workload(n)
    dt = 0.25 * h
    sysm = api.make_system(api.BSSN, n, n, n, h)
    state = torch.from_numpy(st_np).cuda()
    npts = n ** 3

    probe = api.fp64_peak()
    if args.variant is None:
        variant, block, _ = sysm.autotune(state)
    else:
        variant, block = sysm.variant(args.variant)
    jit_s = None
    if not args.no_specialize:
        jit_s = sysm.specialize(True)  # grid, scalars and stage mode compiled in (NVRTC)
    fp64_instr, rhs_flops = sysm.opcount()  # of the body the chosen launch shape runs
    stage_flops = rhs_flops + RK_UPDATE_FLOPS * NVARS  # executed body
    stage_flops_frozen = FROZEN_RHS_FLOPS_BSSN + RK_UPDATE_FLOPS * NVARS
    for _ in range(args.warmup):
        sysm.rk4_step(state, dt, 1)
    torch.cuda.synchronize()

    def barrier():
        if ws > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    # device-resident timed region
    sysm.profile(True)
    sysm.profile_read(reset=True)
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    barrier()
    l0 = api.launch_count()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.steps):
        sysm.rk4_step(state, dt, 1)
    e1.record()
    barrier()
    launches = api.launch_count() - l0
    ms = e0.elapsed_time(e1)
    clk = clocks.stop()
    kern_ms, kern_n = sysm.profile_read(reset=True)
    sysm.profile(False)
    from paper_1410_1764_gb300 import dist as D
    t_max = D.max_over_ranks(ms, device="cuda")
    value = npts * args.steps * ws / (t_max * 1e-3)

    # end to end: host-resident state through the public host-buffer call
    host = torch.from_numpy(st_np).pin_memory()
    nbytes = host.numel() * 8
    for _ in range(2):  # warm-up: the device copy of the state, the step's first launches
        sysm.rk4_step_host(host, dt, 1)
    barrier()
    import gc
    gc.collect()
    gc.disable()  # no Python collection inside the timed calls
    try:
        t0 = time.perf_counter()
        e2e_steps = max(1, min(args.steps, 5))
        per_call = []
        for _ in range(e2e_steps):
            t1 = time.perf_counter()
            sysm.rk4_step_host(host, dt, 1)  # synchronous: copies in, one RK4 step, copies out
            per_call.append((time.perf_counter() - t1) * 1e3)
        barrier()
        e2e_s = time.perf_counter() - t0
    finally:
        gc.enable()
    e2e_v = npts * e2e_steps * ws / e2e_s

    extras = {}
    sms_ = torch.cuda.get_device_properties(local).multi_processor_count
    ISSUE_PEAK[0] = sms_ * 2 * ((clk or {}).get("sm_max_mhz") or 2070.0) * 1e6
    if args.patches_steps > 0:
        extras["patches"] = bench_patches(api, args.patches_steps, npatch=args.patches,
                                          reps=args.patches_reps)  # every rank takes part
    if ws == 1:
        extras["constraints"] = bench_constraints(api, sysm, state, n)
    if ws == 1 and not args.no_adjoint:
        extras["adjoint"] = bench_adjoint(api)
    if ws == 1 and not args.no_wave:
        extras["wave"] = bench_wave(api)
        extras["orders"] = bench_orders(api)
        extras["amr"] = bench_amr(api)
        extras["amr_bssn"] = bench_amr_bssn(api)
    if rank != 0:
        if ws > 1:
            torch.distributed.destroy_process_group()
        return 0

    props = torch.cuda.get_device_properties(local)
    sms = props.multi_processor_count
    max_mhz = (clk or {}).get("sm_max_mhz") or 2070.0
    peak = sms * 2 * 2 * max_mhz * 1e6 / 1e12  # 2 FP64 FMA/clk/SM x 2 flop
    achieved = stage_flops_frozen * npts * kern_n / (kern_ms * 1e-3) / 1e12 if kern_n else None
    achieved_body = stage_flops * npts * kern_n / (kern_ms * 1e-3) / 1e12 if kern_n else None
    # the same launches counted in FP64 instructions (every one an fma) against
    # the pipe's 2 per clock per SM: the ALU-bound fraction of an fma stream
    stage_instr = fp64_instr + NVARS * 2.75  # RK update: 2, 3, 3, 3 fmas per variable over the stages
    issue = stage_instr * npts * kern_n / (kern_ms * 1e-3) if kern_n else None
    issue_peak = sms * 2 * max_mhz * 1e6
    roof = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
            "frac": (achieved / peak) if achieved else None,
            "frac_frozen_F": (achieved / peak) if achieved else None,
            "frac_body_F": (achieved_body / peak) if achieved_body else None,
            "frozen_F_rhs": FROZEN_RHS_FLOPS_BSSN, "body_F_rhs": rhs_flops,
            "flops_basis": "frac/achieved: frozen F (direct-DAG count %d + RK update %.0f per point-stage); "
                           "frac_body_F: the executed body's own count" % (FROZEN_RHS_FLOPS_BSSN,
                                                                          RK_UPDATE_FLOPS * NVARS),
            "traffic": _profile_traffic(kernel_source_hash()),
            "kernel": _kernel_name(api, fp64_instr, variant, jit_s is not None),
            "specialised": jit_s is not None, "jit_compile_s": jit_s,
            "variant": variant, "block": list(block), "fp64_instr_per_point_rhs": fp64_instr, "kernel_ms_avg": kern_ms / kern_n if kern_n else None,
            "flops_per_point_per_stage": stage_flops_frozen,
            "body_flops_per_point_per_stage": stage_flops,
            "fp64_instr_per_point_per_stage": stage_instr,
            "fp64_issue_frac": (issue / issue_peak) if issue else None,
            "peak_basis": "%d SMs x 2 FP64 FMA/clk/SM x 2 flop x %.0f MHz (of derived)" % (sms, max_mhz),
            "fp64_probe_tflops": probe / 1e12,
            "algorithmic_bytes_per_launch": 4.0 * NVARS * 8 * npts}
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": t_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (seeded flat space + U(-1e-10,1e-10) noise)",
            "config": _config(n, ws),
            "e2e": {"value": e2e_v, "unit": UNIT, "h2d_bytes_per_step": nbytes,
                    "d2h_bytes_per_step": nbytes,
                    "ms_per_call_min_median_max": [min(per_call), statistics.median(per_call), max(per_call)],
                    "note": "chemora_rk4_step_host, pinned host state, %d steps; value from their total "
                            "wall time" % e2e_steps},
            "gpu_launches": launches, "roofline": roof, "clocks": clk}
    line.update(extras)
    if ws == 1 and not args.no_cpu_baseline:
        line["parity"] = parity_check(sysm, state, h)
        line["cpu_baseline"] = cpu_baseline(n)
    print(json.dumps(line), flush=True)
    if ws > 1:
        torch.distributed.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="chemora", choices=["chemora", "reference"])
    ap.add_argument("--n", type=int, default=N_DEFAULT, help=argparse.SUPPRESS)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--variant", type=int, default=None,
                    help="force a launch shape of the BSSN stage kernel instead of autotuning")
    ap.add_argument("--no-specialize", action="store_true",
                    help="keep the ahead-of-time stage kernels (no run-time specialisation)")
    ap.add_argument("--no-adjoint", action="store_true")
    ap.add_argument("--no-wave", action="store_true")
    ap.add_argument("--patches-steps", type=int, default=50,
                    help="RK4 steps per schedule and repeat for the batched-patch comparison (0 = skip)")
    ap.add_argument("--patches-reps", type=int, default=5,
                    help="repeats of each schedule (alternating) for the batched-patch comparison")
    ap.add_argument("--patches", type=int, default=64,
                    help="number of patches of the batched-patch comparison (64: the configured workload)")
    ap.add_argument("--wave-only", action="store_true",
                    help="only the two scalar-wave workloads (a profiling entry point; no bench line)")
    ap.add_argument("--adjoint-only", action="store_true",
                    help="only the adjoint workload (a profiling entry point; no bench line)")
    ap.add_argument("--wave-cases", default="32,256",
                    help="scalar-wave workloads of --wave-only (32, 256 or both)")
    ap.add_argument("--orders-only", action="store_true",
                    help="only the finite-difference-order workloads (a profiling entry point; no bench line)")
    ap.add_argument("--amr-only", action="store_true",
                    help="only the two-level BSSN workload (a profiling entry point; no bench line)")
    ap.add_argument("--amr-steps", type=int, default=2, help=argparse.SUPPRESS)
    ap.add_argument("--amr-reps", type=int, default=3, help=argparse.SUPPRESS)
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.wave_only:
        return run_wave_only(args.wave_cases.split(","))
    if args.amr_only:
        return run_amr_only(args.amr_steps, args.amr_reps)
    if args.orders_only:
        import torch
        torch.cuda.set_device(0)
        from paper_1410_1764_gb300 import api
        print(json.dumps({"orders": bench_orders(api)}), flush=True)
        return 0
    if args.adjoint_only:
        return run_adjoint_only()
    return run_chemora(args)


def run_wave_only(cases):
    """The 32^3 plane-wave and/or 256^3 pulse workloads alone, one JSON line
    of their figures (the entry point of the wave kernels' ncu summaries)."""
    import torch
    torch.cuda.set_device(0)
    from paper_1410_1764_gb300 import api
    print(json.dumps({"wave": bench_wave(api, cases)}), flush=True)
    return 0


def run_amr_only(steps, reps):
    """The two-level BSSN workload alone, one JSON line of its figures (the
    entry point of the mesh-refinement kernels' ncu summary)."""
    import torch
    torch.cuda.set_device(0)
    from paper_1410_1764_gb300 import api
    print(json.dumps({"amr_bssn": bench_amr_bssn(api, steps=steps, reps=reps)}), flush=True)
    return 0



def run_adjoint_only():
    """The variable-speed wave adjoint workload alone, one JSON line of its
    figures (the entry point of the adjoint kernels' ncu summary)."""
    import torch
    torch.cuda.set_device(0)
    from paper_1410_1764_gb300 import api
    print(json.dumps({"adjoint": bench_adjoint(api)}), flush=True)
    return 0


if __name__ == "__main__":
    sys.exit(main())
