#!/usr/bin/env python3
"""Benchmark of the Split Bregman self-repelling snake hot path on GB300.

One step = one outer iteration of Alg. 1 (S = 3 semi-implicit inner steps of
Eq. (37), each with the repulsion window sum and the FFT solve of Eqs.
(31)-(33), then the w update of Eqs. (41), (42), (40) and the Bregman update
of Eq. (23)) over the whole image.  Metric: Mpixel.iter/s = H * W * steps /
seconds.

Default workload: the 2048 x 2048 six-ellipse scene (ribbons 3 px, gaps 2 px,
noise 0.1, window l = R = d = 4), the size at which the HBM-roofline target
is stated.  Inputs are resident in HBM when the timed region starts; L2 is
flushed between timed steps outside the timed events: a 256 MiB write, then a
256 MiB read of a second buffer, so that the write's dirty lines are written
back before the step starts instead of inside it.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--workload NAME]
  python bench.py --impl reference ...   # the FP64 CPU oracle on host cores

Under torchrun (N > 1) every rank runs an independent replica (the method has
no cross-image exchange); value = all ranks' pixel-iterations / max time.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = ("SR Mpixel·iter/s (% HBM peak); s per converged mask, plain vs "
          "learned+batched")
UNIT = "Mpixel·iter/s"

# Algorithmic bytes per pixel of each kernel class over one outer iteration
# (S = 3 inner steps; FP32 planes; the Bregman variable is carried as
# e = b - w; w and g are read only on tiles that hold narrow-band pixels,
# which are not counted):
#   prep:      step 1 reads psi, e1, e2 and writes G and div e (20 B); steps 2
#              and 3 read psi and div e and write G (12 B each)
#   rowfft:    read G (4 B), write the half spectrum (4 B), 3 launches
#   colsolve:  read and write the half spectrum (8 B), 3 launches
#   rowifft:   read the half spectrum (4 B) and psi (4 B), write psi (4 B), 3 launches
#   wb_update: read phi, w1, w2, e1, e2 (20 B), write w1, w2, e1, e2 (16 B), 1 launch
BYTES_PER_ITER_PX = {"prep": 44, "rowfft": 24, "colsolve": 24, "rowifft": 36, "wb_update": 36}
LAUNCHES_PER_ITER = {"prep": 3, "rowfft": 3, "colsolve": 3, "rowifft": 3, "wb_update": 1}
KERNEL_NAMES = {"prep": "k_prep", "rowfft": "k_rowfft", "colsolve": "k_colsolve2",
                "rowifft": "k_rowifft", "wb_update": "k_wb_update"}
# column schedule 8 (small images): one kernel per inner step reads G and psi
# and writes phi (12 B/px), in the colsolve class; no row-pass launches
BYTES_PER_ITER_PX_SMALL = {"prep": 44, "colsolve": 36, "wb_update": 36}


# resident iterations (sr_set_resident): one launch per sr_iterate call loads
# phi, w1, w2, e1, e2, g (24 B/px) and stores phi, w1, w2, e1, e2 (20 B/px);
# everything else stays in the cluster's shared memory
BYTES_PER_ITER_PX_RESIDENT = {"resident": 44}


def _kernel_tables(schedule, resident=False):
    """Algorithmic bytes per pixel and iteration, launches per iteration and
    kernel names of the solve path the schedule selects."""
    if resident:
        return dict(BYTES_PER_ITER_PX_RESIDENT), {"resident": 1}, {"resident": "k_resident"}
    names = dict(KERNEL_NAMES)
    if schedule.get("col_schedule") == 7:
        names["colsolve"] = "k_colsolve_rec"
    if schedule.get("col_schedule") == 8:
        names["colsolve"] = "k_solve_small"
        return dict(BYTES_PER_ITER_PX_SMALL), {k: LAUNCHES_PER_ITER[k] for k in
                                               BYTES_PER_ITER_PX_SMALL}, names
    return dict(BYTES_PER_ITER_PX), dict(LAUNCHES_PER_ITER), names


def _peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def _kernel_source_hash() -> str:
    h = hashlib.sha256()
    for name in ("sr_kernels.cu", "sr_fft.cu", "sr_colrec.cu", "sr_tma.cuh", "sr_internal.h",
                 "sr_dft.cuh", "sr_point.cuh"):
        with open(os.path.join(ROOT, "paper_2003_12693_gb300", "csrc", name), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def _ncu_traffic(kernel: str, workload: str):
    """DRAM bytes per launch from the committed ncu summary, if it was taken
    on the current kernel source and the same workload; else None."""
    path = os.path.join(ROOT, "profiles", "ncu_traffic.json")
    if not os.path.exists(path):
        return None
    with open(path) as fh:
        d = json.load(fh)
    e = d.get(workload, {}).get(kernel)
    if not e or e.get("source_hash") != _kernel_source_hash():
        return None
    return float(e["dram_bytes_per_launch"])


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 100 ms."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap,"
              "clocks.mem")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines: list[str] = []
        self.thread = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
            time.sleep(0.3)
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc is not None:
            time.sleep(0.15)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.thread.join(timeout=2)

    def summary(self):
        sm, mx, reasons, mem = [], None, set(), []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx = float(parts[2])
            except ValueError:
                continue
            for name, val in zip(names, parts[5:9]):
                if val.lower() == "active":
                    reasons.add(name)
            if len(parts) > 9:
                try:
                    mem.append(float(parts[9]))
                except ValueError:
                    pass
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm),
                "mem_mhz": statistics.median(mem) if mem else None}


# ----------------------------------------------------------------------------
# CPU oracle legs
# ----------------------------------------------------------------------------
def _oracle_rate(f, phi0, params: dict, budget_s: float, min_iters: int = 1):
    """Time the FP64 oracle as it stands on the host cores: whole outer
    iterations until the time budget is used.  Returns (Mpixel.iter/s, iters, s)."""
    import numpy as np

    import oracle
    p = oracle.Params.from_dict(params)
    g = oracle.edge(f)
    st = oracle.initial_state(phi0)
    H, W = f.shape
    iters, t0 = 0, time.perf_counter()
    while True:
        oracle.iterate(st, g, 1, p)
        iters += 1
        el = time.perf_counter() - t0
        if iters >= min_iters and el >= budget_s:
            break
    del np
    return H * W * iters / el / 1e6, iters, el


def _cores() -> int:
    return int(os.environ.get("OMP_NUM_THREADS") or os.cpu_count() or 1)


def run_reference(args, wl, rank: int, world: int):
    if rank != 0:
        return
    from paper_2003_12693_gb300 import synth  # noqa: F401
    f, phi0 = wl.image(), wl.phi0()
    params = wl.params()
    # per-step sample: one outer iteration on the largest centred crop that keeps
    # the whole run within about two minutes
    per_step = 120.0 / max(1, args.steps + args.warmup)
    import numpy as np

    import oracle
    p = oracle.Params.from_dict(params)
    crop = 128
    t = _time_crop(f, phi0, p, 128)
    for c in (256, 512, 1024, 2048, 4096):
        if c > min(wl.H, wl.W):
            break
        est = t * (c / 128) ** 2 * (1.0 + np.log2(c / 128) / 7.0)
        if est > per_step:
            break
        crop = c
    i0, j0 = (wl.H - crop) // 2, (wl.W - crop) // 2
    fc = np.ascontiguousarray(f[i0:i0 + crop, j0:j0 + crop])
    pc = synth.inset_rect_sdf(crop, crop)
    g = oracle.edge(fc)
    st = oracle.initial_state(pc)
    for _ in range(args.warmup):
        oracle.iterate(st, g, 1, p)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle.iterate(st, g, 1, p)
    el = time.perf_counter() - t0
    value = crop * crop * args.steps / el / 1e6
    sample = (f"one outer iteration (S=3) per step on a centred {crop}x{crop} crop of the "
              f"{wl.name} workload with its own inset-rectangle init, FP64 oracle")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000.0 * el / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {"workload": wl.name, "H": wl.H, "W": wl.W, "R": wl.R,
                                        "d": wl.d, "S": 3, "crop": crop},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": _cores(), "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def _time_crop(f, phi0, p, c):
    import numpy as np

    import oracle
    from paper_2003_12693_gb300 import synth
    fc = np.ascontiguousarray(f[:c, :c])
    st = oracle.initial_state(synth.inset_rect_sdf(c, c))
    g = oracle.edge(fc)
    t0 = time.perf_counter()
    oracle.iterate(st, g, 1, p)
    return time.perf_counter() - t0


# ----------------------------------------------------------------------------
# GPU arm
# ----------------------------------------------------------------------------
def batched_sample(stream, n_images: int = 256, iters: int = 100) -> dict:
    """Many small images in one graph (sr_group_*) against the same images one
    after another.  Height and width drawn independently (seed 3) from the
    31 sides 64, 96, ..., 1024; sides that are not powers of two run the
    mixed-radix FFT passes.  Each image is a crop of one 1024^2 six-ellipse
    scene, inset-rectangle start, R = d = 4."""
    import numpy as np
    import torch

    from paper_2003_12693_gb300 import sr, synth

    rng = np.random.default_rng(3)
    sides = list(range(64, 1025, 32))
    # one 1024^2 six-ellipse scene, each image its top-left H x W crop
    scene = synth.ellipse_scene(1000, H=1024, W=1024, scale=2.0).astype(np.float32)
    ctxs, P = [], 0
    for k in range(n_images):
        H, W = int(rng.choice(sides)), int(rng.choice(sides))
        img_d = torch.from_numpy(np.ascontiguousarray(scene[:H, :W])).cuda()
        phi_d = torch.from_numpy(synth.inset_rect_sdf(H, W).astype(np.float32)).cuda()
        c = sr.Context(H, W, sr.make_params(win_radius=4, d=4.0), stream)
        c.edge_function(img_d)
        c.set_phi(phi_d)
        ctxs.append(c)
        P += H * W
    grp = sr.Group(ctxs)
    lanes = grp.tune()
    grp.iterate(10)
    for c in ctxs:
        c.iterate(2)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    grp.iterate(iters)
    e1.record(stream)
    torch.cuda.synchronize()
    t_group = e0.elapsed_time(e1) / 1e3
    e0.record(stream)
    for c in ctxs:
        c.iterate(iters)
    e1.record(stream)
    torch.cuda.synchronize()
    t_seq = e0.elapsed_time(e1) / 1e3
    grp.close()
    for c in ctxs:
        c.close()
    return {"images": n_images, "pixels": P, "sides": "64, 96, ..., 1024", "iterations": iters,
            "value": P * iters / t_group / 1e6, "unit": UNIT,
            "one_by_one": P * iters / t_seq / 1e6, "speedup": t_seq / t_group,
            "lanes": lanes,
            "how": "sr_group_iterate: one CUDA graph per parity, members' iterations as "
                   "child graphs on concurrent lanes (count chosen by sr_group_tune); "
                   "one_by_one = sr_iterate per "
                   "image in turn; CUDA events on the stream, no L2 flush (state "
                   f"about {P * 14 * 4 / 1e9:.1f} GB)"}


def batched_small_sample(stream, n_images: int = 64, iters: int = 100) -> dict:
    """Many small images (64 of the 128^2 two-disk workload) as one group:
    through the group's graphs, and with every member resident (one cluster
    launch for all of them).  CUDA events on the stream, no L2 flush."""
    import numpy as np
    import torch

    from paper_2003_12693_gb300 import sr, synth

    wl = synth.WORKLOADS["two_disks_128"]
    f = torch.from_numpy(wl.image().astype(np.float32)).cuda()
    phi0 = torch.from_numpy(wl.phi0().astype(np.float32)).cuda()
    out = {"images": n_images, "size": f"{wl.H}x{wl.W}", "iterations": iters, "unit": UNIT}
    for mode in ("graph", "resident"):
        ctxs = []
        for _ in range(n_images):
            c = sr.Context(wl.H, wl.W, sr.make_params(win_radius=wl.R, d=wl.d), stream)
            if mode == "resident":
                c.set_resident(True, cluster=8)  # more images at once than 16-CTA clusters
            c.edge_function(f)
            c.set_phi(phi0)
            ctxs.append(c)
        grp = sr.Group(ctxs)
        grp.tune()
        grp.iterate(4)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        grp.iterate(iters)
        e1.record(stream)
        torch.cuda.synchronize()
        out[mode] = n_images * wl.H * wl.W * iters / (e0.elapsed_time(e1) / 1e3) / 1e6
        grp.close()
        for c in ctxs:
            c.close()
    out["how"] = ("sr_group_iterate: graph = one CUDA graph per parity with the members' "
                  "iterations as child graphs on tuned lanes; resident = every member "
                  "set resident with 8-CTA clusters, all in one launch of one cluster "
                  "per image")
    return out


def resident_sample(stream, wl, iters: int = 100, reps: int = 5) -> dict | None:
    """Whole-run launches with the state resident in one cluster's shared
    memory (sr_set_resident) against the default path, both as a user runs
    many iterations: sr_iterate(iters) per call, CUDA events, no L2 flush
    (the state is L2-sized).  None where the image size does not allow it."""
    import numpy as np
    import torch

    from paper_2003_12693_gb300 import sr

    out = {}
    for resident in (True, False):
        ctx = sr.Context(wl.H, wl.W, sr.make_params(win_radius=wl.R, d=wl.d), stream)
        if resident:
            try:
                ctx.set_resident(True)
            except sr.SRError as e:
                ctx.close()
                if e.status == sr.SR_EUNSUPPORTED:
                    return None
                raise
        ctx.edge_function(torch.from_numpy(wl.image().astype(np.float32)).cuda())
        ctx.set_phi(torch.from_numpy(wl.phi0().astype(np.float32)).cuda())
        ctx.iterate(iters)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            ctx.iterate(iters)
        e1.record(stream)
        torch.cuda.synchronize()
        us = e0.elapsed_time(e1) * 1e3 / (reps * iters)
        out["resident" if resident else "default"] = {
            "us_per_iteration": us, "value": wl.H * wl.W / us, "unit": UNIT}
        ctx.close()
    out["how"] = (f"sr_iterate({iters}) per call, {reps} calls after one untimed call; resident: "
                  "one launch per call, the state in one cluster's shared memory; default: the "
                  "graph of 13 launches per iteration")
    return out


def warm_start_net_sample(stream, H: int = 256, W: int = 256, B: int = 32,
                          steps: int = 20) -> dict:
    """The warm-start network (include/sr_net.h) at its configured size: one
    training step (forward, loss, backward, Adam) and one forward pass on a
    batch of B images, CUDA events on the stream.  Algorithmic work: the six
    3x3 convolutions' 2 * pixels * Cout * 9 * Cin multiply-adds forward, twice
    that backward (input and weight gradients), with the real channel counts
    (the padded first and last layers' extra products are not counted)."""
    import numpy as np
    import torch

    from paper_2003_12693_gb300 import sr_net, synth

    net = sr_net.Net(H, W, max_batch=B, phi_clip=4.0, stream=stream)
    layers = sr_net.layers()
    net.set_params(torch.from_numpy(synth.net_init(1, layers).astype(np.float32)).cuda())
    rng = np.random.default_rng(0)
    f = torch.from_numpy(rng.uniform(0, 1, (B, H, W)).astype(np.float32)).cuda()
    phi = torch.from_numpy(rng.normal(0, 3, (B, H, W)).astype(np.float32)).cuda()
    div = [1, 2, 4, 4, 2, 1]    # resolution divisor of each layer's output
    fwd = sum(2.0 * B * (H // d) * (W // d) * ci * co * 9 for (ci, co), d in zip(layers, div))
    # the first layer needs no input gradient
    bwd = 2 * fwd - 2.0 * B * H * W * layers[0][0] * layers[0][1] * 9
    for _ in range(3):
        net.train_step(f, phi, 1e-4)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    net.kernel_launches(reset=True)
    e0.record(stream)
    for _ in range(steps):
        net.train_step(f, phi, 1e-4)
    e1.record(stream)
    torch.cuda.synchronize()
    t_train = e0.elapsed_time(e1) / steps / 1e3
    launches = net.kernel_launches() / steps
    e0.record(stream)
    for _ in range(steps):
        net.forward(f)
    e1.record(stream)
    torch.cuda.synchronize()
    t_fwd = e0.elapsed_time(e1) / steps / 1e3
    net.close()
    peak = None
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as fh:
            peak = float(json.load(fh)["bf16_tflops"])
    tr_tf = (fwd + bwd) / t_train / 1e12
    fw_tf = fwd / t_fwd / 1e12
    return {"images": B, "H": H, "W": W, "layers": layers, "dtype": "bf16 operands, fp32 accumulate",
            "train_step_ms": t_train * 1e3, "forward_ms": t_fwd * 1e3,
            "train_images_per_s": B / t_train, "forward_images_per_s": B / t_fwd,
            "train_tflops": tr_tf, "forward_tflops": fw_tf,
            "peak_bf16_tflops": peak,
            "frac_train": None if peak is None else tr_tf / peak,
            "frac_forward": None if peak is None else fw_tf / peak,
            "kernel_launches_per_train_step": launches,
            "how": "mma.sync m16n8k16 implicit-GEMM convolutions (cp.async, ldmatrix); "
                   "peak = measured cuBLAS bf16 (burst)"}


def _band_tile_share(ctx, band_width: float) -> dict:
    """Share of the 32 x 32 tiles that hold narrow-band pixels (|phi| < l + eps,
    the tiles on which the window sums and the g, w loads run) at the state
    the timed steps ended in; the step's cost depends on it."""
    import numpy as np
    phi = ctx.get_phi().cpu().numpy()
    H, W = phi.shape
    band = np.abs(phi) < band_width
    t = band[:H // 32 * 32, :W // 32 * 32].reshape(H // 32, 32, W // 32, 32).any(axis=(1, 3))
    return {"tiles": int(t.size), "band_tiles": int(t.sum()), "share": float(t.mean()),
            "band_pixels_share": float(band.mean())}


def job_rate(local_ms: float, units_per_rank: float, world: int, device) -> tuple[float, float]:
    """Whole-job throughput of ``world`` replicas: the slowest rank's time (max
    over ranks, one all-reduce) and the units all ranks processed per second
    of that time.  Returns (max ms, units / s)."""
    import torch
    import torch.distributed as dist

    t = torch.tensor([float(local_ms)], dtype=torch.float64, device=device)
    if world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    ms = float(t.item())
    return ms, world * units_per_rank / (ms / 1e3)


def run_gpu(args, wl, rank: int, world: int, local_rank: int):
    import numpy as np
    import torch
    import torch.distributed as dist

    from paper_2003_12693_gb300 import build, sr

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    if rank == 0:
        build.build()
    if world > 1:
        dist.barrier()
    f = np.ascontiguousarray(wl.image().astype(np.float32))
    phi0 = np.ascontiguousarray(wl.phi0().astype(np.float32))
    params = sr.make_params(win_radius=wl.R, d=wl.d)
    stream = torch.cuda.current_stream()
    ctx = sr.Context(wl.H, wl.W, params, stream)
    resident = False
    if args.resident != "off":
        try:
            ctx.set_resident(True)
            resident = True
        except sr.SRError as e:
            if args.resident == "on" or e.status != sr.SR_EUNSUPPORTED:
                raise
    f_d = torch.from_numpy(f).to(dev)
    phi0_d = torch.from_numpy(phi0).to(dev)
    ctx.edge_function(f_d)
    ctx.set_phi(phi0_d)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    flush_rd = torch.ones(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    sink = torch.empty((), dtype=torch.float32, device=dev)

    def flush_l2(v: float):
        flush.fill_(v)
        sink.copy_(flush_rd.sum())  # evicts the dirty lines the write left in L2

    P = wl.H * wl.W
    schedule = ctx.get_schedule()

    # warm-up: the W counted steps (which also build the CUDA graphs), preceded by
    # back-to-back steps for at least --prewarm-s seconds so that the GPU leaves
    # its idle clock state before anything is timed
    t_pre = time.perf_counter()
    prewarm_steps = 0
    while time.perf_counter() - t_pre < args.prewarm_s:
        ctx.iterate(20)
        torch.cuda.synchronize()
        prewarm_steps += 20
    ctx.iterate(args.warmup)
    torch.cuda.synchronize()

    # ---- timed region: K steps, each bracketed by events, L2 flushed between
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ctx.kernel_launches(reset=True)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local_rank) as clk:
        wall0 = time.perf_counter()
        for k in range(args.steps):
            flush_l2(float(k))
            starts[k].record(stream)
            ctx.iterate(1)
            ends[k].record(stream)
        torch.cuda.synchronize()
        wall = time.perf_counter() - wall0
    if world > 1:
        dist.barrier()
    launches = ctx.kernel_launches(reset=True)
    band_tiles = _band_tile_share(ctx, params.band_l + params.eps)
    step_ms = [s.elapsed_time(e) for s, e in zip(starts, ends)]
    total_ms, rate = job_rate(sum(step_ms), P * args.steps, world, dev)
    value = rate / 1e6

    # ---- per-kernel durations: events around every launch (no graph), minus
    # the cost of the event pair itself (the library's empty kernel between
    # the same event pair); the remainders are then scaled to the graph step
    # (the graph overlaps each kernel's launch with its predecessor's tail), so
    # that the classes add up to ms_per_step
    ctx.profile_enable(True)
    for k in range(args.steps):
        flush_l2(float(k))
        ctx.iterate(1)
    bytes_px, launches_it, names = _kernel_tables(schedule, resident)
    ktimes = {name: ctx.kernel_times(name) for name in bytes_px}
    ctx.kernel_times("reduce")
    ctx.profile_enable(False)
    event_overhead_us = ctx.profile_overhead_us()
    hbm_peak, peak_kind = _peaks()
    kstats = {}
    step_us = 1e3 * total_ms / args.steps
    net = {name: max(1e3 * ms / max(n, 1) - event_overhead_us, 0.05) for name, (ms, n) in ktimes.items()}
    net_sum = sum(net[name] * launches_it[name] for name in net)
    scale = step_us / net_sum if net_sum else 1.0
    for name, (ms, n) in ktimes.items():
        ev_us = 1e3 * ms / max(n, 1)
        in_graph_us = net[name] * scale
        bytes_launch = bytes_px[name] * P / launches_it[name]
        kstats[name] = {"launches": n, "event_avg_us": ev_us, "avg_us": in_graph_us,
                        "share": in_graph_us * launches_it[name] / step_us,
                        "algorithmic_bytes_per_launch": bytes_launch,
                        "achieved_gbs": bytes_launch / (in_graph_us * 1e-6) / 1e9}
    dom = max(kstats, key=lambda k: kstats[k]["share"] or 0)
    ach = kstats[dom]["achieved_gbs"]
    roofline = {"bound": "hbm", "kernel": names[dom], "achieved": ach, "peak": hbm_peak,
                "unit": "GB/s", "frac": ach / hbm_peak, "peak_kind": peak_kind,
                "traffic": _ncu_traffic(names[dom], wl.name)}
    roofline["duration"] = ("in-graph estimate: per-kernel CUDA-event average over the timed "
                            "steps minus the event pair's own cost "
                            f"({event_overhead_us:.2f} us, the same pair around an empty kernel), "
                            "scaled so that the classes add up to the graph step")
    if names[dom] == "k_resident":
        roofline["note"] = ("whole outer iterations in one cluster of 8 or 16 CTAs with the state in "
                            "shared memory: bound by the cluster barriers and on-chip latency of "
                            "each phase, not by DRAM (it reads and writes the state once per call)")
    elif names[dom] == "k_solve_small":
        roofline["note"] = ("whole solve of an inner step in one CTA on one SM: bound by that "
                            "CTA's FFT stages, recursion chains and barriers, not by DRAM")
    elif dom in ("rowfft", "colsolve", "rowifft"):
        roofline["note"] = ("FFT pass on the L2-resident half spectrum (16.8 MB at 2048^2): bound by "
                            "instruction issue, shared memory and barriers, not by DRAM; the "
                            "iteration_roofline entry gives the whole iteration against HBM")
    bytes_iter = sum(bytes_px.values())
    it_gbs = bytes_iter * P / (total_ms / 1e3 / args.steps) / 1e9
    iteration_roofline = {"algorithmic_bytes_per_px": bytes_iter, "achieved_gbs": it_gbs,
                          "frac_of_measured_peak": it_gbs / hbm_peak,
                          "frac_of_nominal_8tbs": it_gbs / 8000.0, "kernels": kstats,
                          "kernels_sum_us": sum(v["avg_us"] * launches_it[k]
                                                for k, v in kstats.items()),
                          "event_overhead_us": event_overhead_us,
                          "band_tiles": band_tiles}

    # ---- end to end through the C-ABI with host buffers
    f_h = torch.from_numpy(f).pin_memory()
    phi0_h = torch.from_numpy(phi0).pin_memory()
    mask_h = torch.empty((wl.H, wl.W), dtype=torch.uint8).pin_memory()
    e2e_iters = args.steps
    jobs = 2
    ctx.segment_host(f_h, phi0_h, 2, 0.0, mask_h)  # warm path
    torch.cuda.synchronize()
    e2e_ms = 0.0
    for _ in range(jobs):
        flush.fill_(0.0)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ctx.segment_host(f_h, phi0_h, e2e_iters, 0.0, mask_h)
        e2e_ms += (time.perf_counter() - t0) * 1e3
    _, e2e_rate = job_rate(e2e_ms, P * e2e_iters * jobs, world, dev)
    e2e_value = e2e_rate / 1e6
    e2e = {"value": e2e_value, "unit": UNIT,
           "h2d_bytes_per_step": (f.nbytes + phi0.nbytes) / e2e_iters,
           "d2h_bytes_per_step": P / e2e_iters,
           "job": f"sr_segment_host: copy image and phi0 from pinned host memory, edge "
                  f"function, {e2e_iters} iterations, mask back to host; per-step bytes "
                  f"amortised over the job"}
    ctx.close()

    if rank != 0:
        return
    batched = None if args.no_batched else batched_sample(stream)
    batched_small = None
    if not args.no_batched and world == 1:
        try:
            batched_small = batched_small_sample(stream)
        except Exception as e:  # a side sample: report, do not lose the line
            batched_small = {"error": f"{type(e).__name__}: {e}"}
    resident_runs = resident_sample(stream, wl) if world == 1 else None
    wsnet = None if args.no_net else warm_start_net_sample(stream)
    cpu = None
    if not args.no_cpu_baseline and world == 1:
        rate, iters, el = _oracle_rate(f.astype(np.float64), phi0.astype(np.float64),
                                       wl.params(), budget_s=args.cpu_budget)
        cpu = {"value": rate, "unit": UNIT, "cores": _cores(), "kind": "oracle",
               "sample": f"{iters} outer iteration(s) (S=3) of the full {wl.H}x{wl.W} "
                         f"workload, {el:.1f} s, FP64 C oracle with OpenMP"}
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": wl.name, "H": wl.H, "W": wl.W, "R": wl.R, "d": wl.d, "S": 3,
                   "description": wl.description,
                   "l2": "flushed between timed steps, outside the events: 256 MiB write, "
                         "then 256 MiB read (no dirty flush lines left in L2)",
                   "parallelism": "replicas" if world > 1 else "single GPU",
                   "fft_schedule": schedule, "resident": resident},
        "roofline": roofline,
        "iteration_roofline": iteration_roofline,
        "cpu_baseline": cpu,
        "e2e": e2e,
        "batched": batched,
        "batched_small": batched_small,
        "resident_runs": resident_runs,
        "warm_start_net": wsnet,
        "gpu_launches": launches,
        "prewarm": {"seconds": args.prewarm_s, "steps": prewarm_steps},
        "clocks": clk.summary(),
        "wall_s_timed_region": wall,
        "step_ms_first_last": [[round(x, 4) for x in step_ms[:5]], [round(x, 4) for x in step_ms[-5:]]],
    }
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--workload", default="ellipses_2048")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batched", action="store_true",
                    help="skip the many-small-images sample (sr_group_*)")
    ap.add_argument("--no-net", action="store_true",
                    help="skip the warm-start network timing sample (sr_net_*)")
    ap.add_argument("--net-only", action="store_true",
                    help="print only the warm-start network sample (profiling runs)")
    ap.add_argument("--net-steps", type=int, default=20)
    ap.add_argument("--cpu-budget", type=float, default=12.0)
    ap.add_argument("--resident", default="off", choices=["auto", "on", "off"],
                    help="time the steps with sr_set_resident (whole iterations in one cluster "
                         "launch) where the image size allows it (auto), always (on: fail "
                         "otherwise) or never (off; the line's resident_runs key compares "
                         "the two paths on many-iteration calls where the size allows)")
    ap.add_argument("--prewarm-s", type=float, default=1.0,
                    help="untimed back-to-back steps before the warm-up steps (clock ramp)")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")

    from paper_2003_12693_gb300 import synth
    wl = synth.WORKLOADS[args.workload]
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, wl, rank, world)
        return
    if args.net_only:
        import torch

        from paper_2003_12693_gb300 import build
        torch.cuda.set_device(local_rank)
        build.build()
        print(json.dumps(warm_start_net_sample(torch.cuda.current_stream(),
                                               steps=args.net_steps)), flush=True)
        return
    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(local_rank)
        os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
        dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))
    try:
        run_gpu(args, wl, rank, world, local_rank)
    finally:
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()


if __name__ == "__main__":
    main()
