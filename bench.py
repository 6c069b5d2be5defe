#!/usr/bin/env python3
"""Benchmark of the fused RC-LBM collide-and-stream step on GB300.

Workload (default): lid-driven square cavity on a rectangular lattice,
2048 x 8192 cells at a = dy/dx = 0.25 (physical aspect 1), c_s^2 = 0.04,
lid speed 0.05, Re = 1000, FP32 deviation storage, timed from a developed
state (a seeded smooth flow of the lid's magnitude, then warm-up steps).  One
benchmark step is one lattice time step over the whole grid (one launch of
the step kernel).  Metric: MLUPS (million lattice-cell updates per second),
whole job, with the state resident in HBM.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

prints one JSON line.  With --impl reference the FP64 CPU oracle is timed
instead, on a bounded sample of the same workload.  Under torchrun (N > 1)
each rank runs an independent replica (the solver does not shard across
GPUs); rank 0 prints.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

BYTES_PER_CELL = {32: 72, 64: 144}   # 9 loads + 9 stores of the storage type
FALLBACK_HBM_GBS = 6800.0


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=50)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--nx", type=int, default=2048)
    ap.add_argument("--ny", type=int, default=8192)
    ap.add_argument("--precision", type=int, default=32, choices=[32, 64])
    ap.add_argument("--e2e-chunk", type=int, default=100,
                    help="lattice steps per end-to-end call sequence")
    ap.add_argument("--e2e-steps", type=int, default=5)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--mask", action="store_true",
                    help="the main workload with the solid mask of the with_mask line")
    ap.add_argument("--no-mask", action="store_true",
                    help="skip the same cavity with a solid mask")
    ap.add_argument("--no-peaks", action="store_true",
                    help="skip the repo's own copy-bandwidth and FP64-FMA measurements")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--no-batch", action="store_true",
                    help="skip the batched-sweep measurements")
    ap.add_argument("--batch-only", action="store_true",
                    help="run only the batched-sweep throughput (for profiling)")
    ap.add_argument("--batch-count", type=int, default=512)
    ap.add_argument("--batch-steps", type=int, default=200)
    ap.add_argument("--batch-shape", default="",
                    help="BX,ROWS: a fixed launch shape instead of the autotuner's")
    ap.add_argument("--ttr-count", type=int, default=64)
    ap.add_argument("--ttr-max-steps", type=int, default=60000)
    ap.add_argument("--no-warm", action="store_true",
                    help="skip the learned warm-start measurement")
    ap.add_argument("--warm-train", type=int, default=2000)
    ap.add_argument("--warm-n", type=int, default=64,
                    help="cavity size n x n of the warm-start instances")
    ap.add_argument("--warm-test", type=int, default=1000,
                    help="held-out warm-start instances")
    ap.add_argument("--warm-only", action="store_true",
                    help="print only the warm-start measurement")
    ap.add_argument("--warm-epochs", type=int, default=80)
    ap.add_argument("--warm-coarse", type=int, default=1,
                    help="network grid this many times coarser than the instances "
                         "(predictions prolonged on the GPU)")
    ap.add_argument("--nn-only", action="store_true",
                    help="only the surrogate's forward and training-step times")
    ap.add_argument("--nn-prof", action="store_true",
                    help="with --nn-only: two forward passes of a one-level 256-channel "
                         "network on 16 instances of 64 x 64 (a case for ncu)")
    ap.add_argument("--config4-ttr", action="store_true",
                    help="only the time to R <= 1e-8 of the full 512-lattice sweep under a "
                         "step cap, batched against sequential (minutes)")
    ap.add_argument("--ttr-cap", type=int, default=20000)
    ap.add_argument("--block-x", type=int, default=0)
    ap.add_argument("--bands", type=int, default=0)
    return ap.parse_args()


def with_obstacles(wl):
    """The cavity with seeded solid rectangles (the masked workload)."""
    from paper_2103_02119_gb300 import workloads as W
    return wl.with_(mask=W.random_obstacles(wl.nx, wl.ny, seed=3, coverage=0.016))


def workload(args):
    from paper_2103_02119_gb300 import workloads as W
    wl = W.cavity(args.nx, args.ny, 0.25, 0.04, 0.05, 1000.0)
    return with_obstacles(wl) if getattr(args, "mask", False) else wl


def workload_config(args, wl):
    return {
        "workload": f"lid-driven cavity {wl.nx}x{wl.ny} cells, a=0.25, Re=1000, "
                    f"lid u=0.05, FP{args.precision} storage"
                    + (", seeded solid rectangles (link mask)" if wl.mask is not None else ""),
        "nx": wl.nx, "ny": wl.ny, "cells": wl.cells, "a": wl.a, "cs2": wl.cs2,
        "lid_u": 0.05, "Re": 1000, "nu": wl.info["nu"],
        "layout": "SoA 9 planes, two buffers, pull streaming",
        "l2": "inputs larger than L2 (state of %d MB per buffer vs 129 MB L2), no flush"
              % (9 * wl.cells * (args.precision // 8) // 2 ** 20),
        "start": "developed: seeded smooth random flow (|u| ~ 0.03, rho - 1 ~ 2e-3), "
                 "then the warm-up steps",
        "parallelism": "replicas" if args.gpus > 1 else "single GPU",
    }


# ------------------------------------------------------------------ clocks --

class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons while running."""

    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device: int):
        self.device = device
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.device), f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "50"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
            time.sleep(0.3)
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc:
            time.sleep(0.1)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.t.join(timeout=2)

    def summary(self):
        if not self.proc:
            return None
        rows = []
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                rows.append((float(parts[0]), float(parts[1]), parts[4:8]))
            except ValueError:
                continue
        if not rows:
            return None
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for _, _, r in rows for i, v in enumerate(r)
                          if v.lower() == "active"})
        return {"sm_mhz": statistics.median(r[0] for r in rows),
                "sm_max_mhz": max(r[1] for r in rows), "reasons": reasons,
                "samples": len(rows)}


# --------------------------------------------------------------- roofline --

def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return FALLBACK_HBM_GBS, "fallback"


STEP_KERNEL_SOURCES = ("rc_step.cu", "rc_free_step.cu", "rnr_step.cu", "step_block.cuh",
                       "lbm_device.cuh")


def step_kernel_hash(csrc=None):
    """Hash of the step kernels' code (comments and whitespace left out, so
    that only a change of the code itself invalidates recorded counters)."""
    import re
    csrc = csrc or os.path.join(ROOT, "paper_2103_02119_gb300", "csrc")
    h = hashlib.sha256()
    for f in STEP_KERNEL_SOURCES:
        with open(os.path.join(csrc, f)) as fh:
            code = fh.read()
        code = re.sub(r"/\*.*?\*/", " ", code, flags=re.S)
        code = re.sub(r"//[^\n]*", " ", code)
        h.update(" ".join(code.split()).encode())
    return h.hexdigest()[:16]


def profiled(precision, key, mask=False):
    """A per-cell figure of the committed ncu summary of the step kernel
    (with a solid mask: its own entry), or None when the kernel has changed
    since it was captured."""
    path = os.path.join(ROOT, "profiles", "rc_step_traffic.json")
    try:
        with open(path) as fh:
            d = json.load(fh)
    except (OSError, ValueError):
        return None
    e = d.get(f"fp{precision}" + ("_mask" if mask else ""))
    if not e or e.get("kernel_sha") != step_kernel_hash():
        return None
    return e.get(key)


def profiled_traffic(precision, cells, mask=False):
    """DRAM bytes per launch from the committed ncu summary, scaled to this
    grid, or None when the kernel has changed since it was captured."""
    b = profiled(precision, "dram_bytes_per_cell", mask)
    return None if b is None else b * cells


def repo_peaks(stream):
    """The roofs measured by the library's own kernels: device-to-device copy
    of 2 GiB buffers (well above the L2) and the FP64 FMA rate."""
    from paper_2103_02119_gb300 import lbm
    copy = lbm.lbm_peak_copy_gbs(2 << 30, 20, stream)
    dfma = lbm.lbm_peak_fp64_gflops(20000, stream)
    return {"copy_gbs": copy, "fp64_gflops": dfma,
            "note": "library kernels: 16-byte-word grid-stride copy between two 2 GiB "
                    "buffers (GB/s = read + write); 8 independent DFMA chains per thread "
                    "(an FMA counts two flops)"}


# ------------------------------------------------------- multi-rank timing --

def max_over_ranks(secs: float, dist=None) -> float:
    """Wall time of the job: the slowest rank's time (every rank runs a
    replica of the workload; there is no data-path collective)."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return secs
    import torch
    t = torch.tensor([secs], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ------------------------------------------------------------- GPU timing --

def developed_start(lat, wl, seed=21):
    from paper_2103_02119_gb300 import workloads as W
    r, u, v = W.smooth_random_fields(wl.nx, wl.ny, seed=seed, u_amp=0.03, rho_amp=2e-3)
    lat.init_fields(r, u, v)


def time_steps(lat, torch, steps, warmup, barrier):
    stream = torch.cuda.current_stream()
    lat.step(warmup)
    torch.cuda.synchronize()
    barrier()
    torch.cuda.synchronize()
    l0 = lat.launch_count
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    lat.step(steps)
    e1.record(stream)
    torch.cuda.synchronize()
    barrier()
    return e0.elapsed_time(e1) / 1e3, lat.launch_count - l0


def e2e(lat, wl, torch, chunk, reps):
    """Through the public API with host buffers: upload the initial fields
    from pinned host memory, advance `chunk` steps, read the fields back."""
    import numpy as np
    N = wl.cells
    pin = [torch.empty(N, dtype=torch.float64).pin_memory() for _ in range(6)]
    host = [t.numpy() for t in pin]
    host[0][:] = 1.0
    host[1][:] = 0.0
    host[2][:] = 0.0
    lat.init_fields(host[0], host[1], host[2])
    lat.step(2)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    from paper_2103_02119_gb300 import lbm
    for _ in range(reps):
        lat.init_fields(host[0], host[1], host[2])
        lat.step(chunk)
        lbm.lbm_moments(lat.h, N, host[3], host[4], host[5])
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    assert np.isfinite(host[3]).all()
    return {"value": N * chunk * reps / dt / 1e6, "unit": "MLUPS",
            "h2d_bytes_per_step": 3 * N * 8, "d2h_bytes_per_step": 3 * N * 8,
            "chunk_lattice_steps": chunk,
            "note": "one e2e step = lbm_init_fields from pinned host rho/u, "
                    f"lbm_step({chunk}), lbm_moments to pinned host rho/u"}


# ------------------------------------------------------------ batched sweep --

def batch_throughput(torch, count, steps, fixed_shape=None):
    """One persistent launch per step over `count` uneven lattices, against
    the same lattices advanced one after another with the single-lattice
    step (one launch per lattice and step)."""
    from paper_2103_02119_gb300 import workloads as W
    from paper_2103_02119_gb300.lbm import Batch, Lattice
    stream = torch.cuda.current_stream()
    ws = W.batch_sweep(count, seed=0)
    cells = sum(w.cells for w in ws)
    b = Batch(ws, stream=stream)
    if fixed_shape:
        b.set_shape(*fixed_shape)
        shape = b.shape
    else:
        shape = b.tune(trial_steps=10)
    b.step(4)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    l0 = b.launch_count
    e0.record(stream)
    b.step(steps)
    e1.record(stream)
    torch.cuda.synchronize()
    tb = e0.elapsed_time(e1) / 1e3
    launches = b.launch_count - l0
    b.close()
    lats = [Lattice.from_workload(w, precision=32, stream=stream) for w in ws]
    for lat in lats:
        lat.step(2)
    torch.cuda.synchronize()
    e0.record(stream)
    for lat in lats:
        lat.step(steps)
    e1.record(stream)
    torch.cuda.synchronize()
    ts = e0.elapsed_time(e1) / 1e3
    for lat in lats:
        lat.close()
    return {"workload": f"{count} channel/cavity lattices, nx, ny log-uniform in [64, 1024], "
                        "a in [0.2, 1], Re log-uniform in [100, 5000], <= 10% obstacles, "
                        "seed 0", "cells": cells, "steps": steps,
            "shape": {"block_x": shape[0], "rows_per_band": shape[1]},
            "batched_mlups": cells * steps / tb / 1e6, "batched_launches": launches,
            "sequential_mlups": cells * steps / ts / 1e6,
            "sequential_launches": count * steps, "speedup": ts / tb}


def batch_time_to_residual(torch, count, max_steps, tol=1e-8, check=100):
    """Wall time until every lattice of a reduced sweep has a steady
    residual <= tol: the batch (autotune + run with retirement) against the
    same lattices run one after another (lbm_step / lbm_diagnostics loop)."""
    import numpy as np
    from paper_2103_02119_gb300 import workloads as W
    from paper_2103_02119_gb300.lbm import Batch, Lattice
    stream = torch.cuda.current_stream()
    ws = W.batch_sweep(count, seed=1, n_range=(16, 32), re_range=(10.0, 100.0))
    b = Batch(ws, stream=stream)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    b.tune(trial_steps=5)
    st, res = b.run(tol, check_every=check, max_steps=max_steps)
    tb = time.perf_counter() - t0
    nb = int(sum(1 for r in res if 0 <= r <= tol))
    steps_b = [b.step_count(k) for k in range(count)]
    b.close()
    ts = 0.0
    ns, steps_s = 0, []
    for w in ws:
        lat = Lattice.from_workload(w, precision=32, stream=stream)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        lat.diagnostics()
        n, R = 0, -1.0
        while n < max_steps:
            lat.step(check)
            n += check
            _, d = lat.diagnostics()
            R = d[4]
            if not np.isfinite(R) or 0 <= R <= tol:
                break
        ts += time.perf_counter() - t0
        ns += int(0 <= R <= tol)
        steps_s.append(n)
        lat.close()
    return {"sample": f"{count} lattices of the same sweep recipe with nx, ny in [16, 32] "
                      "and Re in [10, 100] (seed 1), so that all converge in a bounded run",
            "tol": tol, "check_every": check, "max_steps": max_steps,
            "batched_s": tb, "batched_converged": nb, "batched_max_steps": max(steps_b),
            "sequential_s": ts, "sequential_converged": ns,
            "sequential_max_steps": max(steps_s), "speedup": ts / tb}


def config4_time_to_residual(torch, count=512, cap=20000, tol=1e-8, check=100):
    """The full batched sweep (the batch_throughput recipe, seed 0) from rest
    to R <= tol under a cap of `cap` steps per lattice: the batch (autotune +
    run with retirement) against the same lattices one after another (an
    lbm_step / lbm_diagnostics loop each).  Lattices not converged at the cap
    are listed with their last residual."""
    import numpy as np
    from paper_2103_02119_gb300 import workloads as W
    from paper_2103_02119_gb300.lbm import Batch, Lattice
    stream = torch.cuda.current_stream()
    ws = W.batch_sweep(count, seed=0)
    b = Batch(ws, stream=stream)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    shape = b.tune(trial_steps=5)
    st, res = b.run(tol, check_every=check, max_steps=cap)
    tb = time.perf_counter() - t0
    steps_b = [b.step_count(k) for k in range(count)]
    b.close()
    conv_b = [bool(0 <= r <= tol) for r in res]
    ts, res_s, steps_s = 0.0, [], []
    for w in ws:
        lat = Lattice.from_workload(w, precision=32, stream=stream)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        lat.diagnostics()
        n, R = 0, -1.0
        while n < cap:
            lat.step(check)
            n += check
            st, d = lat.diagnostics()
            R = float("nan") if st != 0 else d[4]
            if not np.isfinite(R) or 0 <= R <= tol:
                break
        ts += time.perf_counter() - t0
        res_s.append(float(R))
        steps_s.append(n)
        lat.close()
    conv_s = [bool(0 <= r <= tol) for r in res_s]
    unstable = [k for k in range(count) if not (np.isfinite(res[k]) and np.isfinite(res_s[k]))]
    cells = sum(w.cells for w in ws)
    return {"sample": f"all {count} lattices of the sweep (seed 0), {cells} cells, rest start",
            "tol": tol, "check_every": check, "cap_steps": cap,
            "shape": {"block_x": shape[0], "rows_per_band": shape[1]},
            "batched_s": tb, "batched_converged": sum(conv_b),
            "batched_lattice_steps": int(sum(steps_b)),
            "sequential_s": ts, "sequential_converged": sum(conv_s),
            "sequential_lattice_steps": int(sum(steps_s)),
            "speedup": ts / tb, "unstable": unstable,
            "not_converged": [{"k": k, "nx": ws[k].nx, "ny": ws[k].ny,
                               "Re": round(ws[k].info["Re"], 1), "kind": ws[k].info["kind"],
                               "R_batched": float(res[k]), "R_sequential": res_s[k]}
                              for k in range(count) if not (conv_b[k] and conv_s[k])]}


def surrogate_times(prof_only=False):
    """Wall time of the surrogate's forward pass and of one Adam training step
    (synchronous calls through the C ABI, host inputs) for the warm-start
    network and a one-level 256-channel network, 16 instances of 64 x 64."""
    import numpy as np
    from paper_2103_02119_gb300 import lbm as L
    rng = np.random.default_rng(0)
    if prof_only:
        nn = L.lbm_nn_create([256], 16, 64, 64, seed=0)
        x = rng.standard_normal((16, 64, 64, 4)).astype(np.float32)
        L.lbm_nn_forward(nn, x)
        L.lbm_nn_forward(nn, x)
        L.lbm_nn_destroy(nn)
        return {"prof": "two forward passes of [256] at 16 x 64 x 64"}
    out = {}
    for channels in ([32, 64, 128, 256], [256]):
        n, hw = 16, 64
        nn = L.lbm_nn_create(channels, n, hw, hw, seed=0)
        x = rng.standard_normal((n, hw, hw, 4)).astype(np.float32)
        x[..., 0] = rng.random((n, hw, hw)) > 0.9
        t = rng.standard_normal((n, hw, hw, 3)).astype(np.float32)
        fl = (x[..., 0] < 0.5).astype(np.uint8)
        for _ in range(3):
            L.lbm_nn_forward(nn, x)
            L.lbm_nn_train_step(nn, x, t, fl, 1e-4)
        t0 = time.perf_counter()
        for _ in range(20):
            L.lbm_nn_forward(nn, x)
        tf = (time.perf_counter() - t0) / 20
        t0 = time.perf_counter()
        for _ in range(20):
            L.lbm_nn_train_step(nn, x, t, fl, 1e-4)
        tt = (time.perf_counter() - t0) / 20
        out[str(channels)] = {"instances": f"{n} x {hw} x {hw}", "forward_ms": tf * 1e3,
                              "train_step_ms": tt * 1e3}
        L.lbm_nn_destroy(nn)
    return out


# ------------------------------------------------------------ small lattice --

def small_lattice(torch):
    """Config 1 (Poiseuille channel, 32 x 32, a = 0.5, FP64, 5,000 steps):
    a lattice this small is bound by latency.  By default lbm_step runs it on
    the cluster kernel (up to 1024 steps per launch); against it, the
    row-band kernel with runs of 50 steps replayed from a CUDA graph, and
    with one call per step."""
    from paper_2103_02119_gb300 import lbm
    from paper_2103_02119_gb300 import workloads as W
    from paper_2103_02119_gb300.lbm import Lattice
    stream = torch.cuda.current_stream()
    wl = W.poiseuille(ny=32, nx=32, a=0.5, cs2=0.16, nu=0.1, U=0.01)
    out = {"workload": "Poiseuille channel 32x32, a=0.5, nu=0.1, FP64", "steps": 5000}
    for mode in ("cluster", "graph", "per_call"):
        lat = Lattice.from_workload(wl, precision=64, stream=stream)
        if mode != "cluster":
            lbm.lbm_set_small_path(lat.h, False)
        lat.step(100)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        if mode != "per_call":
            lat.step(5000)
        else:
            for _ in range(5000):
                lat.step(1)
        e1.record(stream)
        torch.cuda.synchronize()
        out[f"{mode}_us_per_step"] = e0.elapsed_time(e1) * 1e3 / 5000
        lat.close()
    return out


# -------------------------------------------------------- config 2 lattices --

def config2_throughput(torch, steps=200):
    """Config 2's lattices (2048 x 1024, fully periodic, Taylor-Green vortex,
    u0 = 0.02, nu = 1e-2, c_s^2 = 1/3 at a = 1 and 0.3 a^2 below): the step
    in FP32 and FP64 at each aspect ratio, from the seeded initial field."""
    from paper_2103_02119_gb300 import workloads as W
    from paper_2103_02119_gb300.lbm import Lattice
    stream = torch.cuda.current_stream()
    out = {"workload": "Taylor-Green vortex 2048x1024, fully periodic, u0=0.02, nu=1e-2",
           "steps": steps}
    for a in (0.25, 0.5, 1.0):
        cs2 = 1 / 3 if a == 1.0 else 0.3 * a * a
        wl = W.taylor_green(2048, 1024, a, cs2, 1e-2, u0=0.02, seed=0, wavelength=256)
        for prec in (32, 64):
            lat = Lattice.from_workload(wl, precision=prec, stream=stream)
            n = steps if prec == 32 else max(20, steps // 10)
            lat.step(5)
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            lat.step(n)
            e1.record(stream)
            torch.cuda.synchronize()
            out[f"a{a}_fp{prec}_mlups"] = wl.cells * n / (e0.elapsed_time(e1) / 1e3) / 1e6
            lat.close()
    return out


# ---------------------------------------------------------------- warm start --

def warm_start_measure(torch, ntrain, epochs, n=32, ntest=32, coarse=1):
    """Trains the surrogate on steady cavities from the batched solver, then
    runs held-out instances to R <= 1e-8 from the rest state and from the
    network's prediction (both as one batch each).  coarse > 1: the network
    works on a grid that many times coarser (block-averaged inputs and
    targets) and its predictions are prolonged to the instances' grid."""
    import numpy as np
    from paper_2103_02119_gb300 import warmstart as WS
    stream = torch.cuda.current_stream()
    t0 = time.perf_counter()
    wls, x, t, fl, _ = WS.build_dataset(ntrain, seed=0, n=n, stream=stream)
    t_data = time.perf_counter() - t0
    ws = WS.WarmStart([32, 64, 128, 256], n=n // coarse, max_batch=32, seed=0, stream=stream)
    t0 = time.perf_counter()
    hist = ws.train(*WS.coarsen(x, t, fl, coarse), epochs=epochs, lr=2e-3, lr_final=2e-4)
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t0
    test = WS.cavity_set(ntest, seed=1, n=n)
    tx = WS.inputs_of(test)
    t0 = time.perf_counter()
    y = ws.predict_fine(tx, WS.fluid_of(test), coarse)
    t_pred = time.perf_counter() - t0
    rest = WS.solve(test, stream=stream)
    warm = WS.solve(test, inits=[WS.fields_of(w, y[k]) for k, w in enumerate(test)],
                    stream=stream)
    tt = np.stack([WS.targets_of(w, *rest["mean_fields"][k]) for k, w in enumerate(test)])
    m = WS.fluid_of(test)[..., None].astype(bool)
    rms = float(np.sqrt(((y - tt) ** 2 * m).sum() / (3 * m.sum())))
    ws.close()
    ok = [k for k in range(ntest) if 0.0 <= rest["residual"][k] <= 1e-8
          and 0.0 <= warm["residual"][k] <= 1e-8]
    # do the two starts end in the same steady state?  max |u_warm - u_rest|
    # over the fluid, in units of the lid speed (two-step mean fields)
    du = [max(float(np.abs(warm["mean_fields"][k][c] - rest["mean_fields"][k][c]).max())
              for c in (1, 2)) / test[k].info["U"] for k in ok]
    ratio = warm["steps"][ok] / np.maximum(rest["steps"][ok], 1)
    return {"instances": f"{n}x{n} lid-driven cavities with obstacles, a in [0.5, 1], "
                         "Re in [20, 200], seeded; train seed 0, test seed 1",
            "network": "4-level conv encoder-decoder, 32-256 channels, BF16 tcgen05 (TMEM accumulator)"
                       + (f", on a {n // coarse}x{n // coarse} grid, predictions prolonged x{coarse}"
                          if coarse > 1 else ""),
            "train_instances": len(wls), "epochs": epochs, "final_train_loss": hist[-1],
            "test_instances": ntest, "test_rms_error": rms,
            "data_seconds": t_data, "train_seconds": t_train,
            "predict_seconds": t_pred, "tol": 1e-8,
            "rest_steps_mean": float(rest["steps"].mean()),
            "warm_steps_mean": float(warm["steps"].mean()),
            "rest_seconds": rest["seconds"], "warm_seconds": warm["seconds"] + t_pred,
            "steps_ratio_warm_over_rest": float(warm["steps"].mean() / rest["steps"].mean()),
            "both_converged": len(ok),
            "per_instance_ratio_median": float(np.median(ratio)) if ok else None,
            "warm_slower_instances": int((ratio > 1).sum()),
            "max_du_over_U_warm_vs_rest": max(du) if du else None}


# -------------------------------------------------------------- oracle arm --

def oracle_mlups(wl, rows, seconds, warmup_steps=0, steps=None, nthreads=0):
    """The FP64 oracle as it stands, on all host cores (nthreads = 0) or the
    given number of threads, on the same cavity with `rows` rows; returns
    (MLUPS, threads, steps, sample description)."""
    import oracle
    sub = wl.with_(ny=rows)
    p = oracle.OracleParams.make(sub.nx, sub.ny, sub.a, sub.cs2, sub.omega,
                                 periodic_x=sub.periodic_x, periodic_y=sub.periodic_y,
                                 wall_u=sub.wall_u, nthreads=nthreads)
    o = oracle.Oracle(p)
    if warmup_steps:
        o.step(warmup_steps)
    if steps is None:
        t = time.perf_counter()
        o.step(1)
        one = time.perf_counter() - t
        steps = max(1, min(50, int(seconds / max(one, 1e-6))))
    t = time.perf_counter()
    o.step(steps)
    dt = time.perf_counter() - t
    desc = f"{sub.nx}x{rows} cells of the same cavity parameters, {steps} FP64 oracle steps"
    return sub.cells * steps / dt / 1e6, o.threads, steps, desc, dt


def reference_arm(args, rank, world):
    if rank != 0:
        return
    wl = workload(args)
    # each benchmark step is one oracle step on a 2048 x 64 slab of the cavity
    rows = 64
    mlups, threads, steps, desc, dt = oracle_mlups(
        wl, rows, 0, warmup_steps=args.warmup, steps=max(1, args.steps))
    line = {
        "impl": "reference", "metric": "MLUPS", "value": mlups, "unit": "MLUPS",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": dt / max(1, args.steps) * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": workload_config(args, wl),
        "cpu_baseline": {"value": mlups, "unit": "MLUPS", "cores": threads,
                         "kind": "oracle", "sample": desc},
        "e2e": {"value": mlups, "unit": "MLUPS", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------- main --

def main():
    args = parse()
    rank = int(os.environ.get("RANK", 0))
    world = int(os.environ.get("WORLD_SIZE", 1))
    if args.impl == "reference":
        reference_arm(args, rank, world)
        return

    import torch
    local = int(os.environ.get("LOCAL_RANK", 0))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("gloo")

    def barrier():
        if dist is not None:
            dist.barrier()

    if args.batch_only:
        if rank == 0:
            shape = tuple(int(v) for v in args.batch_shape.split(",")) if args.batch_shape else None
            print(json.dumps(batch_throughput(torch, args.batch_count, args.batch_steps, shape)),
                  flush=True)
        return
    if args.warm_only:
        if rank == 0:
            print(json.dumps(warm_start_measure(torch, args.warm_train, args.warm_epochs,
                                                n=args.warm_n, ntest=args.warm_test,
                                                coarse=args.warm_coarse)), flush=True)
        return
    if args.nn_only:
        if rank == 0:
            print(json.dumps(surrogate_times(args.nn_prof)), flush=True)
        return
    if args.config4_ttr:
        if rank == 0:
            print(json.dumps(config4_time_to_residual(torch, args.batch_count, args.ttr_cap)),
                  flush=True)
        return

    from paper_2103_02119_gb300.lbm import Lattice
    wl = workload(args)
    stream = torch.cuda.current_stream()
    lat = Lattice.from_workload(wl, precision=args.precision, stream=stream,
                                block_x=args.block_x, bands=args.bands)
    # time a developed state, not the rest state: a seeded smooth flow of the
    # lid's magnitude with a density perturbation, so that every stored
    # deviation is non-zero from the first timed step
    developed_start(lat, wl)
    with ClockSampler(local) as clk:
        secs, launches = time_steps(lat, torch, args.steps, args.warmup, barrier)
    secs = max_over_ranks(secs, dist)
    cells = wl.cells
    value = world * cells * args.steps / secs / 1e6
    per_launch = secs / args.steps
    # a solid mask adds its link-mask byte to the algorithmic bytes
    bpc_main = BYTES_PER_CELL[args.precision] + (1 if args.mask else 0)
    algo_bytes = bpc_main * cells
    peak, peak_kind = measured_peaks()
    achieved = algo_bytes / per_launch / 1e9
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak,
                "traffic": profiled_traffic(args.precision, cells, args.mask),
                "peak_kind": peak_kind,
                "kernel": f"rc_step_kernel<fp{args.precision}{', mask' if args.mask else ''}>",
                "algorithmic_bytes_per_cell": bpc_main}
    e2e_res = None if args.no_e2e else e2e(lat, wl, torch, args.e2e_chunk, args.e2e_steps)
    peaks = None
    if rank == 0 and not args.no_peaks:
        peaks = repo_peaks(stream)
        roofline["frac_vs_repo_copy"] = achieved / peaks["copy_gbs"]

    fp64 = None
    if not args.no_fp64 and args.precision == 32:
        lat.close()
        lat64 = Lattice.from_workload(wl, precision=64, stream=stream)
        s64, _ = time_steps(lat64, torch, max(20, args.steps // 20), 5, barrier)
        n64 = max(20, args.steps // 20)
        a64 = BYTES_PER_CELL[64] * cells / (s64 / n64) / 1e9
        fp64 = {"value": cells * n64 / s64 / 1e6, "unit": "MLUPS", "steps": n64,
                "roofline": {"bound": "alu", "hbm_achieved": a64, "hbm_peak": peak,
                             "unit": "GB/s", "hbm_frac": a64 / peak}}
        # the FP64 roof: FP64 instructions per cell counted by ncu (DFMA,
        # DADD, DMUL each take the pipe once) against the FMA rate the
        # library measures (one FMA = two flops); the flop count (DFMA
        # twice) is reported beside it
        ops = profiled(64, "fp64_pipe_ops_per_cell")
        fl = profiled(64, "fp64_flops_per_cell")
        if ops is not None and fl is not None and peaks is not None:
            rate = fp64["value"] * 1e6
            pk = peaks["fp64_gflops"]
            fp64["roofline"].update({
                "fp64_pipe_ops_per_cell": ops, "fp64_flops_per_cell": fl,
                "alu_achieved": rate * ops / 1e9, "alu_peak": pk / 2, "alu_unit": "Gop/s",
                "alu_frac": rate * ops / 1e9 / (pk / 2),
                "alu_flops_achieved": rate * fl / 1e9, "alu_flops_peak": pk,
                "alu_flops_frac": rate * fl / 1e9 / pk})
        lat64.close()
    else:
        lat.close()

    # The same cavity with seeded solid rectangles (a 1.6 % cap on the solid
    # fraction; 0.8 % of the cells at this size and seed): the mask path,
    # whose link-mask byte adds 1 B per cell to the 72 B.
    with_mask = None
    if rank == 0 and not args.no_mask:
        from paper_2103_02119_gb300 import workloads as W
        wm = with_obstacles(wl) if wl.mask is None else wl
        latm = Lattice.from_workload(wm, precision=args.precision, stream=stream)
        nm = max(100, args.steps // 10)
        sm, _ = time_steps(latm, torch, nm, 10, barrier)
        latm.close()
        bpc = BYTES_PER_CELL[args.precision] + 1
        am = bpc * cells / (sm / nm) / 1e9
        with_mask = {"value": cells * nm / sm / 1e6, "unit": "MLUPS", "steps": nm,
                     "solid_fraction": float(wm.mask.mean()),
                     "roofline": {"bound": "hbm", "achieved": am, "peak": peak, "unit": "GB/s",
                                  "frac": am / peak, "algorithmic_bytes_per_cell": bpc,
                                  "traffic": profiled_traffic(args.precision, cells, True)}}

    batch = None
    if rank == 0 and not args.no_batch:
        batch = batch_throughput(torch, args.batch_count, args.batch_steps)
        batch["time_to_residual"] = batch_time_to_residual(torch, args.ttr_count,
                                                           args.ttr_max_steps)

    small = small_lattice(torch) if rank == 0 and not args.no_batch else None
    config2 = config2_throughput(torch) if rank == 0 and not args.no_fp64 else None

    warm = None
    if rank == 0 and not args.no_warm:
        warm = warm_start_measure(torch, args.warm_train, args.warm_epochs, n=args.warm_n,
                                  ntest=args.warm_test, coarse=args.warm_coarse)

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        mlups, threads, steps, desc, _ = oracle_mlups(wl, wl.ny, args.cpu_seconds)
        cpu = {"value": mlups, "unit": "MLUPS", "cores": threads, "kind": "oracle",
               "sample": desc}
        # the same oracle on one thread, on a smaller slab of the cavity
        m1, _, _, d1, _ = oracle_mlups(wl, 256, min(5.0, args.cpu_seconds), nthreads=1)
        cpu["single_thread"] = {"value": m1, "unit": "MLUPS", "cores": 1, "sample": d1}

    if rank == 0:
        line = {
            "metric": "MLUPS", "value": value, "unit": "MLUPS", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": per_launch * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": f"f{args.precision}", "data": "synthetic",
            "config": workload_config(args, wl), "roofline": roofline,
            "cpu_baseline": cpu, "e2e": e2e_res, "gpu_launches": launches,
            "clocks": clk.summary(), "fp64": fp64, "batch": batch, "small_lattice": small,
            "config2": config2,
            "warm_start": warm, "repo_peaks": peaks, "with_mask": with_mask,
        }
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
