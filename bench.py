#!/usr/bin/env python3
"""Particle pushes/s of the GB300 patch-PIC hot path on the 2D LWFA workload.

One "step" is one pass of the whole hot path (work-queue build, particle
interpolation + Boris push + Esirkepov deposition, window injection, particle
exchange, Yee E and B) over the 2048 x 512-cell LWFA window: 4 particles per cell,
a0 = 4 Gaussian laser focused at the foot of a density ramp. The run starts from that
initial condition (plasma from the pulse centre, 1 048 576 particles) and is developed
for 1800 untimed steps: the window is then full of plasma (4.2M particles) and the
wake has formed, so the timed steps see the uneven patch loads of the configured
2000-step run. Prints one JSON line (rank 0), with a bounded served parameter-scan
sample (p50/p99 time to completion, aggregate pushes/s). `--impl reference` times the
FP64 CPU oracle instead.

Timing: W untimed warm-up steps, then K steps between CUDA events on the sim's
stream with a synchronize (and a barrier under torchrun) on both sides; the
working set (particles + fields) is larger than the 129 MB L2.
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
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "particle pushes/s (interp+push+deposit) vs HBM roofline; served p50/p99 sim latency"
UNIT = "pushes/s"
# FP64 dense rate of GB300 from the unit counts and clock (nominal 1.25 TFLOP/s)
FP64_NOMINAL_TFLOPS = 1.25
# Algorithmic FP64 flops of one push (FMA = 2, rsqrt and division 1 each), counted from
# the kernels' no-crossing path.
# 2D: positions 6, shapes 4 x 7, interpolation 6 x 20, Boris 64, move 11, deposition 96
# (new shapes 14, weights and running sums 33, charge factors 4, 21 taps 45). ncu counts
# 371 executed FP64 flops per push: the rsqrt and division iterations and the deposits of
# cell-crossing particles add the rest.
FLOPS_PER_PUSH_2D = 325
# 3D: positions 9, shapes 6 x 7, interpolation 6 x 65, Boris 64, move 15, deposition 222
# (new shapes 21, weights 54, running sums 9, charge factors 3, 54 taps 135).
FLOPS_PER_PUSH_3D = 742
# The 2D FP64 kernel runs most of those flops as exact fixed-point integer arithmetic
# (offsets, shapes, gather, deposit weights and products); the FP64 pipe keeps the Boris
# push and the move, with the internals of rsqrt and the reciprocal: 68 FP64-pipe
# instructions per push (ncu, developed LWFA run). At 2 FP64 lane-operations per clock
# per SM that is this kernel's own ceiling.
FP64_PIPE_INSTR_PER_PUSH_2D = 68
GB300_SMS = 152


DTYPE = {"fp64": "f64", "fp32": "f32", "df64": "f32x2 (double-word, ~48-bit)"}


def _ppc(w, n):
    p = w["params"]
    n = len(w["particles"]["x"]) if n is None else n
    return n / float(np.prod(p["n"][:p["dims"]]))


def bytes_per_push(dt, w, n=None):
    """Algorithmic HBM bytes of the particle kernel per push: particle state read and
    written once, weight read once; E and B^n read once and J (FP64) written once per
    cell, shared by the particles per cell (n particles on the grid: the timed state's
    count; the workload's when None). dt: "fp64", "fp32" or "df64"."""
    dims = w["params"]["dims"]
    es = 4 if dt == "fp32" else 8
    pos = dims * es + (0 if dt == "fp64" else 4)
    return 2 * (pos + 3 * es) + es + (6 * es + 3 * 8) / _ppc(w, n)


def step_bytes_per_push(dt, w, n=None):
    """Algorithmic HBM bytes of a whole step per push: the particle kernel's bytes plus,
    per cell and shared by its particles, the field update's (E, B and the FP64 J read,
    E and B written, the next J zeroed)."""
    es = 4 if dt == "fp32" else 8
    return bytes_per_push(dt, w, n) + (6 * es + 3 * 8 + 6 * es + 3 * 8) / _ppc(w, n)


def step_roofline(dt, w, pushes_per_s, n=None):
    """The whole step's algorithmic bytes per second against the measured HBM peak."""
    hbm = measured_peaks().get("hbm_gbs")
    achieved = step_bytes_per_push(dt, w, n) * pushes_per_s / 1e9
    return {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
            "frac": achieved / hbm if hbm else None,
            "bytes_per_push": step_bytes_per_push(dt, w, n)}
# kernels per step: queue build, push, [window injection], exchange, repack plan and its
# two copy kernels (which return at once unless a patch needs room), Yee E, Yee B, end
def kernels_per_step(window: bool, merge: bool = False, split: bool = False) -> int:
    """Kernels in one captured step: queue build, push, 2 Yee, exchange, repack plan + 2
    copies, end step; injection with the window; the merge kernel and the three split
    kernels (count, id offsets, apply) with load limiting."""
    return (10 if window else 9) + (1 if merge else 0) + (3 if split else 0)


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=300)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="fp64", choices=["fp64", "fp32", "df64"])
    ap.add_argument("--variants", default="fp32,df64",
                    help="other precisions timed in the same run (comma list, or none)")
    ap.add_argument("--nx", type=int, default=2048)
    ap.add_argument("--ny", type=int, default=512)
    ap.add_argument("--chunk", type=int, default=0, help="queue chunk when not autotuned")
    ap.add_argument("--patch", default="", help="patch sides when not autotuned, e.g. 16,8,8")
    ap.add_argument("--merge-above", type=int, default=0,
                    help="load limiting: merge particle groups in patches above this count")
    ap.add_argument("--merge-dp", type=float, default=0.05, help="merge momentum-bin width")
    ap.add_argument("--split-below", type=int, default=0,
                    help="load limiting: split particles of cells holding fewer than this many")
    ap.add_argument("--split-wmin", type=float, default=0.0, help="weight floor of splitting")
    ap.add_argument("--autotune", default="cached", choices=["cached", "on", "off"],
                    help="cached: the layouts recorded in the package's tuning table (measured "
                         "there when missing); on: measure again; off: workload patch, --chunk")
    ap.add_argument("--workload", default="lwfa",
                    choices=["lwfa", "lwfa3d", "stress3d", "thermal", "serve", "batch"])
    ap.add_argument("--requests", type=int, default=256, help="serve: number of requests")
    ap.add_argument("--rate", type=float, default=4.0, help="serve: mean arrivals per second")
    ap.add_argument("--budget-gb", type=float, default=96.0, help="serve: HBM budget")
    ap.add_argument("--batch-sims", type=int, default=16,
                    help="batch: simulations of the scan distribution stepped together")
    ap.add_argument("--mapping", default="queue", choices=["queue", "static"])
    ap.add_argument("--total", type=int, default=64 * 2 ** 20, help="stress3d particles")
    ap.add_argument("--maxwell-order", type=int, default=2, choices=[2, 6],
                    help="field solver: 2 = Yee, 6 = sixth-order staggered differences "
                         "(time step 0.76 of Yee's limit instead of 0.95)")
    ap.add_argument("--lwfa-start", default="ramp", choices=["ramp", "full"],
                    help="lwfa: ramp = the configured initial condition (plasma from the "
                         "pulse centre); full = the window already full of plasma")
    ap.add_argument("--develop", type=int, default=-1,
                    help="untimed steps before the warm-up (-1: 1800 for the lwfa ramp "
                         "start, when the window is full of plasma and the wake has formed; "
                         "0 otherwise)")
    ap.add_argument("--serve-requests", type=int, default=24,
                    help="requests of the bounded serving sample in the default line (0: off)")
    ap.add_argument("--serve-rate", type=float, default=8.0,
                    help="mean arrivals per second of the serving sample")
    ap.add_argument("--no-variant", action="store_true", help="skip the other precision")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--trace-steps", type=int, default=0,
                    help="after the timed runs, step one more sim this many steps and record "
                         "the time per step and the patch-load spread along the run")
    ap.add_argument("--trace-every", type=int, default=100, help="trace window in steps")
    return ap.parse_args()


def develop_steps(args):
    """Untimed steps that bring the workload to the state the timed steps measure."""
    if args.develop >= 0:
        return args.develop
    return 1800 if args.workload == "lwfa" and args.lwfa_start == "ramp" else 0


def capacity_for(w):
    """Particle slots of a sim: three times the largest count the run reaches (the
    window full of plasma for LWFA), twice the count for 3D."""
    p = w["params"]
    n = len(w["particles"]["x"])
    if p["dims"] == 2 and p.get("window"):
        full = p["n"][0] * p["n"][1] * p["inject_ppc"][0] * p["inject_ppc"][1]
        return 3 * max(n, full)
    return 3 * n if p["dims"] == 2 else 2 * n


def workload(nx, ny, kind="lwfa", total=64 * 2 ** 20, order=2, start="full"):
    """The synthetic workload; with the sixth-order solver the time step is 0.76 of
    Yee's limit (the sixth-order scheme is stable below 120/149 = 0.805 of it).
    LWFA `start`: "ramp" = the configured initial condition (plasma from the pulse
    centre, ramp of 64 cells), "full" = the window already full of plasma."""
    from paper_1511_03878_gb300 import inputs

    cfl = 0.76 if order == 6 else 0.95
    if kind == "stress3d":
        # 256x128x128 cells, log-normal counts per 16^3 block, 8^3 patches
        w = inputs.stress3d(total=total, cfl=cfl)
        w["params"] = dict(w["params"], patch=(8, 8, 8))
    elif kind == "thermal":
        w = inputs.thermal2d(seed=1511, cfl=cfl)
    elif kind == "lwfa3d":
        # 512x128x128 window full of plasma, 2 particles per cell (16 777 216)
        w = inputs.lwfa3d(ramp_x0=-8.0, ppc=(2, 1, 1), cfl=cfl)
    elif start == "ramp":
        w = inputs.lwfa2d(nx=nx, ny=ny, cfl=cfl)
    else:
        # the window full of plasma: density ramp placed before x = 0
        w = inputs.lwfa2d(nx=nx, ny=ny, ramp_x0=-8.0, cfl=cfl)
    if order != 2:
        w["params"] = dict(w["params"], maxwell_order=order)
    return w


TRAFFIC_TABLE = os.path.join(ROOT, "profiles", "traffic.md")
# the sources a particle kernel is built from (the digest in the traffic table)
KERNEL_SOURCES = {2: ("k_push2d.cu", "fix62.cuh", "pic_device.cuh", "df64.cuh", "pic_internal.h"),
                  3: ("k_push3d.cu", "fix62.cuh", "pic_device.cuh", "df64.cuh", "pic_internal.h")}


def code_only(text):
    """C/C++/CUDA source without its comments, each whitespace run outside string and
    character literals reduced to one newline (if it holds one) or one space: a comment
    or layout edit leaves it as it was, a change to the code does not. Raw string
    literals and digit separators are not recognised; the kernel sources use neither."""
    out = []
    i, n = 0, len(text)

    def space(nl):
        if out and out[-1] in " \n":
            if nl:
                out[-1] = "\n"
        elif out:
            out.append("\n" if nl else " ")

    while i < n:
        c = text[i]
        if text.startswith("//", i):
            j = text.find("\n", i)
            i = n if j < 0 else j
        elif text.startswith("/*", i):
            j = text.find("*/", i + 2)
            i = n if j < 0 else j + 2
            space(False)
        elif c in "\"'":
            j = i + 1
            while j < n and text[j] != c:
                j += 2 if text[j] == "\\" else 1
            out.append(text[i:j + 1])
            i = j + 1
        elif c.isspace():
            space(c == "\n")
            i += 1
        else:
            out.append(c)
            i += 1
    return "".join(out).strip()


def source_digest(dims, root=None):
    """First 16 hex digits of sha256 over the code of the kernel's sources (code_only)."""
    h = hashlib.sha256()
    for f in KERNEL_SOURCES[dims]:
        with open(os.path.join(root or ROOT, "paper_1511_03878_gb300", "csrc", f)) as fh:
            h.update(code_only(fh.read()).encode())
        h.update(b"\0")
    return h.hexdigest()[:16]


def measured_traffic(kernel, workload_name, patch, chunk, dims):
    """DRAM bytes per launch of `kernel` from the committed ncu summary table, or None
    when no capture matches this workload and layout or the kernel sources changed
    since the capture (their digest differs)."""
    try:
        with open(TRAFFIC_TABLE) as f:
            lines = f.read().splitlines()
    except OSError:
        return None
    digest = source_digest(dims)
    lay = "x".join(str(v) for v in patch)
    for ln in lines:
        cols = [c.strip().strip("`") for c in ln.strip().strip("|").split("|")]
        if len(cols) < 6 or not cols[4].isdigit():
            continue
        if (cols[0] == kernel and cols[1] == workload_name and cols[2] == lay
                and cols[3] == str(chunk) and cols[5] == digest):
            return int(cols[4])
    return None


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except OSError:
        return {}


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled while the timed work runs."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, dev):
        self.dev = dev
        self.rows = []
        self.proc = None
        self.t = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-i", str(self.dev), "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self.t = threading.Thread(target=self._read, daemon=True)
        self.t.start()
        time.sleep(0.3)

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                self.rows.append(parts)

    def stop(self):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
        if self.t:
            self.t.join(timeout=2)

    def summary(self):
        if not self.rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        sm = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in self.rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for r in self.rows:
            for i, nm in enumerate(names):
                if r[5 + i].lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(self.rows)}


def dist_setup(n_gpus):
    """One process per GPU (replicas of the whole simulation, no data-path collective):
    NCCL between GPUs, gloo when there is no GPU (host-side tests of this logic)."""
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch
        import torch.distributed as dist

        dist.init_process_group("nccl" if n_gpus > 1 and torch.cuda.is_available() else "gloo")
    return rank, world, local


def _on_gpu_backend():
    import torch.distributed as dist

    return dist.get_backend() == "nccl"


def barrier(world):
    if world > 1:
        import torch
        import torch.distributed as dist

        if _on_gpu_backend():
            dist.barrier(device_ids=[torch.cuda.current_device()])
        else:
            dist.barrier()


def _reduce(x, world, op):
    if world == 1:
        return x
    import torch
    import torch.distributed as dist

    t = torch.tensor([x], dtype=torch.float64, device="cuda" if _on_gpu_backend() else "cpu")
    dist.all_reduce(t, op=op)
    return float(t.item())


def max_over_ranks(x, world):
    import torch.distributed as dist

    return _reduce(x, world, dist.ReduceOp.MAX if world > 1 else None)


def sum_over_ranks(x, world):
    import torch.distributed as dist

    return _reduce(x, world, dist.ReduceOp.SUM if world > 1 else None)


def job_value(pushes_all_ranks, ms_slowest):
    """Whole-job throughput: the pushes of all ranks over the slowest rank's time."""
    return pushes_all_ranks / (ms_slowest * 1e-3)


def trace_run(args, w, precision, chunk):
    """Time per step and patch-load spread along one long run (ablation of the mapping).

    Every `trace_every` steps: the mean ms per step of that window (CUDA events on the
    sim's stream), max/mean particles per patch at its end, and the particle count. The
    patch-count read syncs between windows, so these rows are not the bench's value."""
    import torch

    from paper_1511_03878_gb300 import binding

    prec = {"fp64": binding.PIC_FP64, "fp32": binding.PIC_FP32, "df64": binding.PIC_DF64}[precision]
    mapping = binding.PIC_MAP_STATIC if args.mapping == "static" else binding.PIC_MAP_QUEUE
    sim = binding.Sim(w["params"], precision=prec, capacity=capacity_for(w), chunk=chunk,
                      mapping=mapping, merge_above=args.merge_above, merge_dp=args.merge_dp,
                      split_below=args.split_below, split_wmin=args.split_wmin)
    rows = []
    try:
        sim.load(w)
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        done = 0
        while done < args.trace_steps:
            k = min(args.trace_every, args.trace_steps - done)
            ev0.record(sim.stream)
            sim.step(k)
            ev1.record(sim.stream)
            ev1.synchronize()
            done += k
            c = sim.patch_counts().astype(np.float64)
            rows.append([done, round(ev0.elapsed_time(ev1) / k, 4),
                         round(float(c.max() / max(c.mean(), 1e-30)), 3), int(c.sum())])
        sim.sync()
    finally:
        sim.close()
    return {"precision": precision, "mapping": args.mapping, "every": args.trace_every,
            "columns": ["step", "ms_per_step", "max_over_mean_patch", "particles"],
            "rows": rows}


def run_gpu(args, w, precision, K, W, world, clocks=None, chunk=0, snapshot=False):
    """Returns timing + roofline of one precision on this rank's GPU (and, with
    `snapshot`, the developed state as a host workload for the end-to-end run)."""
    import torch

    from paper_1511_03878_gb300 import binding

    prec = {"fp64": binding.PIC_FP64, "fp32": binding.PIC_FP32, "df64": binding.PIC_DF64}[precision]
    cap = capacity_for(w)
    mapping = binding.PIC_MAP_STATIC if args.mapping == "static" else binding.PIC_MAP_QUEUE
    sim = binding.Sim(w["params"], precision=prec, capacity=cap, chunk=chunk, mapping=mapping,
                      merge_above=args.merge_above, merge_dp=args.merge_dp,
                      split_below=args.split_below, split_wmin=args.split_wmin)
    sim.load(w)
    counts0 = sim.patch_counts()
    stream = sim.stream
    dev = develop_steps(args)
    if dev > 0:
        sim.step(dev)  # untimed: the run up to the state the timed steps measure
        sim.sync()
    counts_dev = sim.patch_counts().astype(np.float64)
    state = None
    if snapshot:
        # the developed state on the host, for the end-to-end measurement (x in the window
        # frame, B at the half step as the loader takes it)
        q = sim.particles()
        f = sim.fields()
        state = dict(w, particles=q, E=[f["Ex"], f["Ey"], f["Ez"]], B=[f["Bx"], f["By"], f["Bz"]])
    sim.step(W)
    sim.sync()
    counts_t0 = sim.patch_counts().astype(np.float64)
    n0 = sim.num_particles()
    if clocks:
        clocks.start()
    barrier(world)
    torch.cuda.synchronize()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    sim.step(K)
    ev1.record(stream)
    torch.cuda.synchronize()
    barrier(world)
    ms = ev0.elapsed_time(ev1)
    if clocks:
        clocks.stop()
    sim.sync()  # raises on any latched device error
    n1 = sim.num_particles()
    repacks = sim.repacks()
    ms = max_over_ranks(ms, world)
    pushes = K * 0.5 * (n0 + n1)
    pushes_all = sum_over_ranks(pushes, world)
    # per-kernel CUDA-event pass (same kernels, same launch shapes) for the roofline
    prof = sim.profile(K)
    push_ms = prof["push"] / K
    dt = precision
    n_push = 0.5 * (n0 + n1)
    peaks = measured_peaks()
    hbm = peaks.get("hbm_gbs")
    dims = w["params"]["dims"]
    if precision == "fp64":
        fl = FLOPS_PER_PUSH_2D if dims == 2 else FLOPS_PER_PUSH_3D
        achieved = fl * n_push / (push_ms * 1e-3) / 1e12
        roof = {"bound": "alu", "achieved": achieved, "peak": FP64_NOMINAL_TFLOPS,
                "unit": "TFLOP/s", "frac": achieved / FP64_NOMINAL_TFLOPS, "traffic": None,
                "kernel": f"push{dims}d_kernel<double>",
                "peak_source": ("nominal FP64 1.25 TFLOP/s (recipe unit counts x clock), in "
                                "FP64-equivalent flops; the 2D kernel computes most of them "
                                "exactly in fixed point on the integer units, so the fraction "
                                "can exceed 1 (design_bound: its FP64-pipe ceiling)"),
                "hbm_frac_of_measured": (bytes_per_push(dt, w, n_push) * n_push
                                         / (push_ms * 1e-3) / 1e9 / hbm) if hbm else None}
        if dims == 2:
            mhz = (clocks.summary().get("sm_mhz") if clocks else None) or 2070.0
            cap = GB300_SMS * 2 * mhz * 1e6 / FP64_PIPE_INSTR_PER_PUSH_2D
            rate = n_push / (push_ms * 1e-3)
            roof["design_bound"] = {"unit": "FP64 pipe", "fp64_pipe_instr_per_push":
                                    FP64_PIPE_INSTR_PER_PUSH_2D, "sm_mhz": mhz,
                                    "max_pushes_per_s": cap, "kernel_pushes_per_s": rate,
                                    "frac": rate / cap}
    else:
        achieved = bytes_per_push(dt, w, n_push) * n_push / (push_ms * 1e-3) / 1e9
        peak = hbm if hbm else 6800.0
        tname = "float" if precision == "fp32" else "df64"
        roof = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "traffic": None, "kernel": f"push{dims}d_kernel<{tname}>",
                "peak_source": "measured" if hbm else "fallback"}
        if precision == "df64":
            fl = FLOPS_PER_PUSH_2D if dims == 2 else FLOPS_PER_PUSH_3D
            roof["fp64_equivalent_tflops"] = fl * n_push / (push_ms * 1e-3) / 1e12
    # DRAM bytes per launch from the committed ncu capture of this kernel and layout
    roof["traffic"] = measured_traffic(roof["kernel"], config_dict(args, precision)["workload"],
                                       w["params"]["patch"], chunk or 2048, dims)
    roof["traffic_source"] = ("ncu dram__bytes_read.sum + dram__bytes_write.sum per launch "
                              "(profiles/traffic.md)" if roof["traffic"] is not None else
                              "no capture of the current kernel sources in this layout")
    out = dict(ms=ms, pushes=pushes, pushes_all=pushes_all, n=n_push, profile={k: v / K for k, v in prof.items()},
               roofline=roof, push_ms=push_ms, repacks=repacks, state=state,
               timed_state={"developed_steps": dev, "steps_before_timing": dev + W,
                            "particles": int(counts_t0.sum()),
                            "max_over_mean_patch": float(counts_t0.max() / counts_t0.mean()),
                            "max_over_mean_patch_at_load": float(counts0.max() / counts0.mean()),
                            "max_patch": int(counts_t0.max())})
    if args.split_below > 0:
        out["split"] = {"below": args.split_below, "wmin": args.split_wmin,
                        "added": sim.split_count()}
    if args.merge_above > 0:
        counts1 = sim.patch_counts()
        out["merge"] = {"above": args.merge_above, "dp": args.merge_dp,
                        "removed": sim.merged(),
                        "particles_at_load": int(counts0.sum()), "particles_end": int(counts1.sum()),
                        "max_over_mean_at_load": float(counts0.max() / counts0.mean()),
                        "max_over_mean_end": float(counts1.max() / counts1.mean()),
                        "max_patch_at_load": int(counts0.max()), "max_patch_end": int(counts1.max())}
    sim.close()
    del sim
    torch.cuda.empty_cache()
    return out


def pipelined_steps(sim, K):
    """K steps, each with a read of its step record; step k + 1 is enqueued before the
    host waits for step k's record (two record slots, alternating). Returns the records
    (steps taken, window shifts) in step order."""
    recs = []
    for k in range(K):
        sim.step(1)
        sim.step_record_async(k & 1)
        if k:
            recs.append(sim.record_wait((k - 1) & 1))
    if K:
        recs.append(sim.record_wait((K - 1) & 1))
    return recs


def run_e2e(args, w, precision, K, chunk=0, world=1):
    """Same metric through the public C ABI with host buffers, all inside the timed
    region: load the particles and fields from pinned host arrays (H2D), then K steps,
    each followed by a read of its step record (the device step state and status word,
    60 bytes D2H). The reads are pipelined: step k + 1 is enqueued before the host waits
    for step k's record, so the device does not idle between steps. At the end the
    energy and the axis wake field. `w` is the state the device-timed steps start from
    (the developed run)."""
    import torch

    from paper_1511_03878_gb300 import binding

    prec = {"fp64": binding.PIC_FP64, "fp32": binding.PIC_FP32, "df64": binding.PIC_DF64}[precision]
    n = len(w["particles"]["x"])
    sim = binding.Sim(w["params"], precision=prec, capacity=capacity_for(w), chunk=chunk)
    # the inputs sit in page-locked host memory, as a serving process would keep them
    keep = []

    def pinned(a):
        t = torch.empty(a.shape, dtype=torch.from_numpy(np.ascontiguousarray(a)).dtype,
                        pin_memory=True)
        keep.append(t)
        out = t.numpy()
        out[...] = a
        return out

    wp = dict(w, particles={k: pinned(v) for k, v in w["particles"].items()},
              E=[pinned(a) for a in w["E"]], B=[pinned(a) for a in w["B"]])
    torch.cuda.synchronize()
    barrier(world)
    t0 = time.perf_counter()
    sim.load(wp)
    tl = time.perf_counter()
    pipelined_steps(sim, K)
    ts = time.perf_counter()
    e = sim.energy()
    ax = sim.ex_axis()
    t1 = time.perf_counter()
    dims = w["params"]["dims"]
    cfg = sim.cfg
    ncell = cfg.n[0] * cfg.n[1] * (cfg.n[2] if dims == 3 else 1)
    # the loader copies the caller's arrays as they are (FP64 positions, momenta and
    # weights, int32 ids), five per-patch int arrays and the FP64 fields E and B; the
    # device validates, bins, orders, converts, places and pads; the host reads back the
    # per-(patch, bank class) counts and three reductions
    h2d = n * (8 * (dims + 4) + 4) + 6 * ncell * 8 + 5 * sim.npatch * 4 + 24
    d2h = 60 * K + e.nbytes + ax.nbytes + 32 * 4 * sim.npatch + 24
    sim.close()
    seconds = max_over_ranks(t1 - t0, world)
    return dict(value=job_value(sum_over_ranks(n * K, world), 1e3 * seconds), h2d=h2d / K,
                d2h=d2h / K, seconds=seconds,
                split_ms={"load": 1e3 * (tl - t0), "steps": 1e3 * (ts - tl),
                          "readback": 1e3 * (t1 - ts)})


def oracle_sim(w, steps):
    """The FP64 CPU oracle loaded with workload `w`, with particle room for `steps`
    steps of window injection (at most one column of cells per step)."""
    import oracle as orc

    p = w["params"]
    dims = p["dims"]
    c = orc.make_config(dims, p["n"][:dims], p["d"][:dims], p["dt"], window=p["window"],
                        q=p["q"], m=p["m"], n0=p["n0"], ramp_x0=p["ramp_x0"],
                        ramp_len=p["ramp_len"], inject_ppc=p["inject_ppc"],
                        order=p.get("maxwell_order", 2))
    col = (int(np.prod(p["n"][1:dims])) * int(np.prod(p["inject_ppc"][:dims]))
           if p["window"] else 0)
    o = orc.OracleSim(c, len(w["particles"]["x"]) + (steps + 2) * col)
    o.set_particles(w["particles"])
    o.set_fields(w["E"], w["B"])
    return o


def oracle_sample(args, frac):
    """The bench's workload cut to about `frac` of its particles, for a bounded CPU
    timing sample: fewer transverse rows of the window (LWFA, so that the injected
    columns shrink with it), or every k-th particle of the same grid (thermal, 3D
    stress). Returns the workload and a description of the cut."""
    order = args.maxwell_order
    # LWFA: the window full of plasma, the particle count of the developed state the GPU
    # steps are timed on (the oracle cannot be developed 1800 steps in a bounded sample)
    w = workload(args.nx, args.ny, args.workload, args.total, order, start="full")
    if frac >= 1.0:
        return w, "the full workload (window full of plasma)"
    if args.workload == "lwfa":
        ny = max(32, int(args.ny * frac) // 32 * 32)
        return (workload(args.nx, ny, "lwfa", order=order, start="full"),
                f"{args.nx}x{ny} rows of the window full of plasma")
    if args.workload == "lwfa3d":
        from paper_1511_03878_gb300 import inputs

        side = max(16, int(128 * math.sqrt(frac)) // 8 * 8)
        w3 = inputs.lwfa3d(ny=side, nz=side, ramp_x0=-8.0, ppc=(2, 1, 1),
                           cfl=0.76 if order == 6 else 0.95)
        if order != 2:
            w3["params"] = dict(w3["params"], maxwell_order=order)
        return w3, f"512x{side}x{side} cells of the window"
    k = max(1, int(round(1.0 / frac)))
    w = dict(w, particles={key: v[::k].copy() for key, v in w["particles"].items()})
    return w, f"one particle in {k} on the same grid"


def oracle_rate(args, n_full, seconds_budget, max_steps=50, threads=1):
    """Pushes/s of the FP64 CPU oracle (as it stands: its plain step on one thread, or
    its threaded step, identical bit for bit, on `threads`) on a bounded number of
    steps of the same workload (at most 5M particles of it)."""
    w, what = oracle_sample(args, min(1.0, 5e6 / n_full))
    n = len(w["particles"]["x"])
    o = oracle_sim(w, max_steps)
    t0 = time.perf_counter()
    o.step(1, threads=threads)
    t1 = time.perf_counter()
    steps = 1
    budget_steps = int(max(0, min(max_steps - 1, seconds_budget / max(t1 - t0, 1e-6) - 1)))
    pushes = n
    if budget_steps > 0:
        n1 = o.num_particles()
        t2 = time.perf_counter()
        o.step(budget_steps, threads=threads)
        t3 = time.perf_counter()
        steps += budget_steps
        pushes += n1 * budget_steps
        t1 = t1 + (t3 - t2)
    return pushes / (t1 - t0), steps, n, what


def reference_arm(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle as orc

    orc.build()
    threads = os.cpu_count() or 1
    n_full = len(workload(args.nx, args.ny, args.workload, args.total,
                          args.maxwell_order, start="full")["particles"]["x"])
    total = args.steps + args.warmup
    # each step is a bounded sample: a cut of the same workload (at most 5M particles,
    # fewer if K+W steps would exceed about three minutes), timed after one probe step
    frac = min(1.0, 5e6 / n_full)
    w, what = oracle_sample(args, frac)
    o = oracle_sim(w, total)
    t0 = time.perf_counter()
    o.step(1, threads=threads)
    t_step = time.perf_counter() - t0
    done = 1
    need = min(1.0, 180.0 / max(total * t_step, 1e-9))
    if need < 1.0:
        w, what = oracle_sample(args, frac * need)
        o = oracle_sim(w, total)
        done = 0
    n = len(w["particles"]["x"])
    o.step(max(0, args.warmup - done), threads=threads)
    n0 = o.num_particles()
    t0 = time.perf_counter()
    o.step(args.steps, threads=threads)
    el = time.perf_counter() - t0
    n1 = o.num_particles()
    value = args.steps * 0.5 * (n0 + n1) / el
    name = config_dict(args, "fp64")["workload"]
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic (seeded, shaped like the paper's runs)",
        "config": config_dict(args, "fp64"),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle",
                         "sample": f"FP64 C oracle, threaded step (bit-identical to the plain "
                                   f"one) on {threads} host threads, {what} of {name} "
                                   f"({n} particles), {args.steps} steps"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def config_dict(args, precision):
    """The workload (the same for both arms); the launch layout is reported apart."""
    if args.workload == "stress3d":
        base = {"workload": f"stress3d-256x128x128-lognormal1.5-n{args.total}", "grid": [256, 128, 128],
                "dx": 0.1, "particles": args.total}
    elif args.workload == "lwfa3d":
        base = {"workload": "lwfa3d-512x128x128-ppc2-fullwindow", "grid": [512, 128, 128],
                "dx": 0.125, "dy": 0.5, "dz": 0.5, "particles_per_cell": 2, "laser_a0": 4.0}
    elif args.workload == "thermal":
        base = {"workload": "thermal2d-128x128-ppc16", "grid": [128, 128], "dx": 0.1,
                "particles_per_cell": 16}
    elif args.lwfa_start == "ramp":
        dev = develop_steps(args)
        base = {"workload": f"lwfa2d-{args.nx}x{args.ny}-ppc4-from-step{dev}",
                "grid": [args.nx, args.ny], "dx": 0.125, "dy": 0.5, "particles_per_cell": 4,
                "laser_a0": 4.0, "initial_condition": "plasma from the pulse centre, "
                "64-cell ramp (the configured 2000-step run)", "timed_from_step": dev}
    else:
        base = {"workload": f"lwfa2d-{args.nx}x{args.ny}-ppc4-fullwindow",
                "grid": [args.nx, args.ny], "dx": 0.125, "dy": 0.5, "particles_per_cell": 4,
                "laser_a0": 4.0}
    if args.maxwell_order != 2:
        base = dict(base, workload=base["workload"] + f"-maxwell{args.maxwell_order}",
                    maxwell_order=args.maxwell_order, cfl=0.76)
    l2 = ("working set (about 25 MB of particles and fields) fits in the 129 MB L2; steps "
          "run back to back with no flush, so this rate is L2-resident"
          if args.workload == "thermal" else
          "inputs larger than L2 (particles + fields > 129 MB), no flush")
    return {**base, "precision": precision, "l2": l2,
            "parallelism": f"replicas x{args.gpus}" if args.gpus > 1 else "single GPU"}


def launch_layout(args, w, precision):
    """Patch and chunk for one precision: measured by the autotuner, or the workload's
    patch and --chunk. Returns the workload with that patch, the chunk and a record."""
    from paper_1511_03878_gb300 import autotune, binding

    prec = {"fp64": binding.PIC_FP64, "fp32": binding.PIC_FP32, "df64": binding.PIC_DF64}[precision]
    mapping = ("persistent work queue (largest chunk first)" if args.mapping == "queue"
               else "static: one CTA per patch")
    if args.autotune == "off" or args.mapping == "static":
        chunk = args.chunk
        if args.patch:
            w = dict(w, params=dict(w["params"], patch=tuple(int(v) for v in args.patch.split(","))))
        rec = {"patch": list(w["params"]["patch"]), "chunk": chunk or autotune.DEFAULT_CHUNK,
               "mapping": mapping, "autotuned": False}
        return w, chunk, rec
    n = len(w["particles"]["x"])
    cap = 3 * n if w["params"]["dims"] == 2 else 2 * n
    cache = autotune.TUNING_TABLE if args.autotune == "cached" else None
    c = autotune.tune(w, prec, capacity=cap, warmup=10, steps=100, margin=0.03, cache_file=cache)
    rec = {"patch": list(c.patch), "chunk": c.chunk, "mapping": mapping, "autotuned": True,
           "autotune": {"source": "tuning table" if cache else "measured in this run",
                        "candidates": len(c.table), "seconds": round(c.seconds, 1),
                        "ns_per_push": {f"{'x'.join(map(str, p))}/{k}": round(v, 4)
                                        for p, k, v in c.table}}}
    return dict(w, params=dict(w["params"], patch=c.patch)), c.chunk, rec


def batch_arm(args):
    """Batching: simulations of the parameter-scan distribution (mixed grids, particles
    per cell and densities, so very uneven patch loads), FP32, stepped together in one
    persistent particle launch per step (pic_batch) against the same simulations
    stepped one at a time; value = the batched aggregate pushes/s."""
    import torch

    import __graft_entry__
    from paper_1511_03878_gb300 import binding, serve

    __graft_entry__.build()
    torch.cuda.set_device(0)
    reqs = serve.scan_requests(n=args.batch_sims, rate=1.0, seed=1516)
    sims = []
    for r in reqs:
        w = serve.request_workload(r)
        sim = binding.Sim(w["params"], precision=binding.PIC_FP32,
                          capacity=serve.request_capacity(r))
        sim.load(w)
        sims.append(sim)
    for sim in sims:
        sim.sync()
    stream = torch.cuda.Stream()
    handles = [s.h for s in sims]
    nbytes = binding.pic_batch_required_bytes(handles)
    arena = torch.empty(nbytes + 256, dtype=torch.uint8, device="cuda")
    batch = binding.pic_batch_create(handles, (arena.data_ptr() + 255) // 256 * 256, nbytes,
                                     stream.cuda_stream)
    K, W = args.steps, args.warmup
    clocks = ClockSampler(0)
    binding.pic_batch_step(batch, W)
    stream.synchronize()
    n0 = sum(s.num_particles() for s in sims)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    clocks.start()
    ev0.record(stream)
    binding.pic_batch_step(batch, K)
    ev1.record(stream)
    ev1.synchronize()
    clocks.stop()
    ms_batch = ev0.elapsed_time(ev1)
    n1 = sum(s.num_particles() for s in sims)
    pushes_batch = K * 0.5 * (n0 + n1)
    binding.pic_batch_destroy(batch)
    # the same simulations one at a time, each on its own stream and graph
    ms_seq, pushes_seq = 0.0, 0.0
    for sim in sims:
        sim.step(W)
        sim.sync()
        a = sim.num_particles()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(sim.stream)
        sim.step(K)
        e1.record(sim.stream)
        e1.synchronize()
        ms_seq += e0.elapsed_time(e1)
        pushes_seq += K * 0.5 * (a + sim.num_particles())
    for sim in sims:
        sim.sync()
        sim.close()
    value = pushes_batch / (ms_batch * 1e-3)
    seq = pushes_seq / (ms_seq * 1e-3)
    counts = [r.nx * r.ny * r.ppc for r in reqs]
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 1, "steps": K,
        "warmup": W, "ms_per_step": ms_batch / K, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic (seeded LWFA parameter-scan requests)",
        "config": {"workload": f"batched-lwfa-scan-{args.batch_sims}sims",
                   "grids": sorted({f"{r.nx}x{r.ny}" for r in reqs}),
                   "ppc": sorted({r.ppc for r in reqs}), "precision": "fp32",
                   "particles": int(n0), "largest_over_smallest_sim": max(counts) / min(counts),
                   "l2": "inputs larger than L2 in aggregate, no flush"},
        "batching": {"sims": len(reqs), "batched_pushes_per_s": value,
                     "one_at_a_time_pushes_per_s": seq, "batched_over_one_at_a_time": value / seq,
                     "one_at_a_time_ms_per_step": ms_seq / K},
        "gpu_launches": kernels_per_step(True) * K,
        "clocks": clocks.summary(),
    }
    print(json.dumps(line), flush=True)


def serve_sample(args, main_run):
    """A bounded, saturated sample of the served parameter scan (the metric's second
    half): `--serve-requests` requests of the scan distribution arriving at
    `--serve-rate` per second, FP32, admitted by HBM budget and stepped together with
    continuous batching. Returns p50/p99 time to completion, the aggregate pushes/s and
    the ratio to the FP64 single-simulation rate measured above."""
    from paper_1511_03878_gb300 import serve

    reqs = serve.scan_requests(n=args.serve_requests, rate=args.serve_rate, seed=1517)
    serve.Server(budget_bytes=8 << 30).run([serve.Request(rid=0, nx=256, ny=128, a0=3.0,
                                                          n0=0.01, ppc=2, steps=20)])
    srv = serve.Server(budget_bytes=int(args.budget_gb * (1 << 30)), quantum=25)
    res = srv.run(reqs)
    summ = serve.summarize(res)
    fp64 = main_run["pushes"] / (main_run["ms"] * 1e-3) if args.precision == "fp64" else None
    return {**summ, "max_resident": srv.max_resident, "precision": "fp32",
            "rate_per_s": args.serve_rate, "budget_gb": args.budget_gb,
            "distribution": "grids {256x128, 512x256, 1024x256, 2048x512}, a0 U[2,6], "
                            "n0 U[0.003,0.02] n_c, ppc {1,2,4,8}, 500-2000 steps, seed 1517",
            "served_over_fp64_single": (summ["aggregate_pushes_per_s"] / fp64) if fp64 else None}


def serve_arm(args):
    """Served parameter scan: Poisson arrivals, HBM-budget admission, continuous
    batching; value = aggregate pushes/s, with p50/p99 time-to-completion."""
    import torch

    import __graft_entry__
    from paper_1511_03878_gb300 import binding, serve

    __graft_entry__.build()
    torch.cuda.set_device(0)
    reqs = serve.scan_requests(n=args.requests, rate=args.rate)
    # warm-up: one small request through the same server path
    serve.Server(budget_bytes=8 << 30).run([serve.Request(rid=0, nx=256, ny=128, a0=3.0, n0=0.01,
                                                          ppc=2, steps=20)])
    clocks = ClockSampler(0)
    clocks.start()
    srv = serve.Server(budget_bytes=int(args.budget_gb * (1 << 30)), quantum=25)
    res = srv.run(reqs)
    clocks.stop()
    summ = serve.summarize(res)
    # the plain FP64 single-simulation path on the largest scan grid, for comparison
    w = serve.request_workload(serve.Request(rid=0, nx=2048, ny=512, a0=4.0, n0=0.01, ppc=4,
                                             steps=0))
    w = dict(w, particles=workload(2048, 512)["particles"])
    sim = binding.Sim(w["params"], precision=binding.PIC_FP64,
                      capacity=3 * len(w["particles"]["x"]))
    sim.load(w)
    sim.step(3)
    sim.sync()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(sim.stream)
    sim.step(50)
    ev1.record(sim.stream)
    torch.cuda.synchronize()
    fp64_rate = 50 * sim.num_particles() / (ev0.elapsed_time(ev1) * 1e-3)
    sim.close()
    line = {
        "metric": METRIC, "value": summ["aggregate_pushes_per_s"], "unit": UNIT, "n_gpus": 1,
        "steps": int(sum(r.steps for r in reqs)), "warmup": 1,
        "ms_per_step": None, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32", "data": "synthetic (seeded LWFA parameter scan)",
        "config": {"workload": f"served-lwfa-scan-{args.requests}req-{args.rate}per_s",
                   "grids": ["256x128", "512x256", "1024x256", "2048x512"], "a0": [2, 6],
                   "n0": [0.003, 0.02], "ppc": [1, 2, 4, 8], "steps": [500, 2000],
                   "budget_gb": args.budget_gb, "precision": "fp32",
                   "l2": "inputs larger than L2 for the large grids, no flush"},
        "serving": {**summ, "max_resident": srv.max_resident,
                    "fp64_single_sim_pushes_per_s": fp64_rate,
                    "served_over_fp64_single": summ["aggregate_pushes_per_s"] / fp64_rate},
        "clocks": clocks.summary(),
    }
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        reference_arm(args)
        return
    if args.workload == "serve":
        serve_arm(args)
        return
    if args.workload == "batch":
        batch_arm(args)
        return
    import torch

    rank, world, local = dist_setup(args.gpus)
    torch.cuda.set_device(local)
    import __graft_entry__

    if rank == 0:
        __graft_entry__.build()
    barrier(world)
    if rank != 0:
        __graft_entry__.build()

    w = workload(args.nx, args.ny, args.workload, args.total, args.maxwell_order,
                 start=args.lwfa_start)
    # layouts are tuned on the window full of plasma (the grid and particle count of the
    # developed state) and applied to the run from its initial condition
    wt = workload(args.nx, args.ny, args.workload, args.total, args.maxwell_order, start="full")
    clocks = ClockSampler(local)
    others = [] if args.no_variant or args.variants == "none" else [
        v for v in args.variants.split(",") if v and v != args.precision]
    if w["params"]["dims"] == 3:  # the double-word precision is 2D only
        others = [v for v in others if v != "df64"]
    layouts = {}
    for v in [args.precision] + others:
        wl, ch, rec = launch_layout(args, wt, v)
        layouts[v] = (dict(w, params=dict(w["params"], patch=wl["params"]["patch"])), ch, rec)
    wm, chunk_m, _ = layouts[args.precision]
    main_run = run_gpu(args, wm, args.precision, args.steps, args.warmup, world, clocks, chunk_m,
                       snapshot=not args.no_e2e)
    variants = {v: run_gpu(args, layouts[v][0], v, args.steps, args.warmup, world,
                           chunk=layouts[v][1]) for v in others}
    e2e = None
    if not args.no_e2e:
        e2e = run_e2e(args, main_run["state"] or wm, args.precision, args.steps, chunk_m, world)
    main_run["state"] = None
    trace = None
    if rank == 0 and args.trace_steps > 0:
        trace = trace_run(args, wm, args.precision, chunk_m)
    serving = None
    if rank == 0 and args.serve_requests > 0 and args.workload == "lwfa" and world == 1:
        serving = serve_sample(args, main_run)
    cpu = None
    if rank == 0 and not args.no_cpu and world == 1:
        n_full = len(wt["particles"]["x"])
        threads = os.cpu_count() or 1
        rate, steps, n, what = oracle_rate(args, n_full, args.cpu_seconds, threads=threads)
        rate1, steps1, _, _ = oracle_rate(args, n_full, args.cpu_seconds / 2, max_steps=10)
        cpu = {"value": rate, "unit": UNIT, "cores": threads, "kind": "oracle",
               "sample": f"FP64 C oracle, threaded step (bit-identical to the plain one) on "
                         f"{threads} host threads, {steps} steps of {what} of "
                         f"{config_dict(args, 'fp64')['workload']} ({n} particles)",
               "single_thread": {"value": rate1, "cores": 1, "steps": steps1}}
    if rank != 0:
        return
    value = job_value(main_run["pushes_all"], main_run["ms"])
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": main_run["ms"] / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": DTYPE[args.precision],
        "data": "synthetic (seeded LWFA-shaped initial condition, no dataset)",
        "config": config_dict(args, args.precision),
        "launch": layouts[args.precision][2],
        "roofline": main_run["roofline"],
        "roofline_step": step_roofline(args.precision, wm, value, main_run["n"]),
        "cpu_baseline": cpu,
        "e2e": ({"value": e2e["value"], "unit": UNIT,
                 "h2d_bytes_per_step": e2e["h2d"], "d2h_bytes_per_step": e2e["d2h"],
                 "split_ms": e2e["split_ms"]}
                if e2e else None),
        "gpu_launches": kernels_per_step(bool(w["params"].get("window")),
                                         args.merge_above > 0, args.split_below > 0) * args.steps,
        "clocks": clocks.summary(),
        "kernel_ms_per_step": main_run["profile"],
        "particles": main_run["n"],
        "timed_state": main_run["timed_state"],
        "capacity_repacks": main_run["repacks"],
    }
    if serving is not None:
        line["serving"] = serving
    if "merge" in main_run:
        line["merge"] = main_run["merge"]
    if "split" in main_run:
        line["split"] = main_run["split"]
    if trace is not None:
        line["trace"] = trace
    if variants:
        line["variants"] = {v: {
            "value": job_value(r["pushes_all"], r["ms"]),
            "ms_per_step": r["ms"] / args.steps, "roofline": r["roofline"],
            "roofline_step": step_roofline(v, layouts[v][0],
                                           job_value(r["pushes_all"], r["ms"]), r["n"]),
            "kernel_ms_per_step": r["profile"], "dtype": DTYPE[v],
            "capacity_repacks": r["repacks"],
            "launch": layouts[v][2]} for v, r in variants.items()}
    print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()
