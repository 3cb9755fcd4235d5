"""Continuous-batching server for laser-wakefield parameter-scan simulations.

The paper motivates large simulation campaigns over laser and plasma parameters
(Sec. 1: campaigns to explore parameter space; Sec. 2.2: the laser and plasma
parameters of one case). Here many small 2D LWFA simulations share one GPU:

* a request (grid, a0, density, particles per cell, steps) is admitted when its
  arena (``pic_required_bytes``) fits in the free HBM budget; otherwise it waits;
* admitted simulations are prepared (inputs, arena, upload) on a worker thread and
  then stay resident on the device until they finish;
* all resident simulations are stepped together: one ``pic_batch`` whose step graph
  runs a single persistent particle launch over the patches of every simulation,
  so uneven simulations share the SMs through the work queue;
* when a simulation finishes, its diagnostics are read back, its arena is freed and
  the batch is rebuilt at the next step boundary with whatever is resident.

Results are returned per request with arrival, admission and completion times, so
p50/p99 time-to-completion and the aggregate pushes/s can be reported.
"""
from __future__ import annotations

import concurrent.futures as cf
import dataclasses
import math
import threading
import time

import numpy as np

from . import binding, inputs

PPC_LATTICE = {1: (1, 1), 2: (2, 1), 4: (2, 2), 8: (4, 2)}


@dataclasses.dataclass
class Request:
    rid: int
    nx: int
    ny: int
    a0: float
    n0: float
    ppc: int
    steps: int
    arrival: float = 0.0  # seconds after the server starts


def request_workload(r: Request, patch=(32, 32)) -> dict:
    """LWFA input of a scan request: the 2D window and pulse scaled with the box
    (pulse 1/4 of the box from the right edge, duration and waist capped by the box),
    the density ramp starting at the pulse centre."""
    dx, dy = 0.125, 0.5
    Lx, Ly = r.nx * dx, r.ny * dy
    return inputs.lwfa2d(nx=r.nx, ny=r.ny, dx=dx, dy=dy, ppc=PPC_LATTICE[r.ppc], n0=r.n0,
                         ramp_cells=64, a0=r.a0, w0=min(30.0, Ly / 4), tau=min(25.0, Lx / 10),
                         laser_back=Lx / 4, seed=1514 + r.rid, patch=patch)


def request_capacity(r: Request) -> int:
    """Particle slots for a request: the window full of plasma, with headroom."""
    return int(2.5 * r.nx * r.ny * r.ppc) + 4096


def scan_requests(n=256, rate=4.0, seed=1515, steps=(500, 2000),
                  grids=((256, 128), (512, 256), (1024, 256), (2048, 512))) -> list[Request]:
    """The served parameter scan: Poisson arrivals (mean `rate` per second), grids,
    a0 ~ U[2, 6], n0 ~ U[0.003, 0.02], ppc in {1, 2, 4, 8}, steps ~ U{steps}."""
    rng = np.random.default_rng(seed)
    t = 0.0
    out = []
    for i in range(n):
        t += rng.exponential(1.0 / rate)
        g = grids[rng.integers(len(grids))]
        out.append(Request(rid=i, nx=g[0], ny=g[1], a0=float(rng.uniform(2, 6)),
                           n0=float(rng.uniform(0.003, 0.02)),
                           ppc=int(rng.choice([1, 2, 4, 8])),
                           steps=int(rng.integers(steps[0], steps[1] + 1)), arrival=t))
    return out


@dataclasses.dataclass
class Result:
    rid: int
    arrival: float
    admitted: float
    started: float
    completed: float
    steps: int
    pushes: float
    energy: np.ndarray
    ex_axis: np.ndarray
    particles: int
    arena_bytes: int


class _Running:
    def __init__(self, req, sim, nbytes, admitted, started, n0):
        self.req = req
        self.sim = sim
        self.nbytes = nbytes
        self.admitted = admitted
        self.started = started
        self.remaining = req.steps
        self.n_start = n0


class Server:
    def __init__(self, budget_bytes: int, precision: int = binding.PIC_FP32, quantum: int = 25,
                 chunk: int = 0, prep_workers: int = 2, patch=(32, 32)):
        import torch

        self.torch = torch
        self.budget = int(budget_bytes)
        self.precision = precision
        self.quantum = int(quantum)
        self.chunk = chunk
        self.patch = patch
        self.pool = cf.ThreadPoolExecutor(max_workers=prep_workers)
        self.stream = torch.cuda.Stream()
        self.max_resident = 0
        self.timeline = []  # (time, event, rid)

    def _bytes(self, r: Request) -> int:
        w = dict(dims=2, n=(r.nx, r.ny, 1), d=(0.125, 0.5, 1.0), dt=inputs.cfl_dt((0.125, 0.5)),
                 window=True, n0=r.n0, ramp_x0=0.0, ramp_len=8.0, inject_ppc=PPC_LATTICE[r.ppc] + (1,),
                 patch=self.patch)
        cfg = binding.make_config(w, self.precision, request_capacity(r), self.chunk)
        return binding.pic_required_bytes(cfg) + 256

    def _prepare(self, r: Request):
        torch = self.torch
        stream = torch.cuda.Stream()
        with torch.cuda.stream(stream):
            w = request_workload(r, self.patch)
            sim = binding.Sim(w["params"], precision=self.precision,
                              capacity=request_capacity(r), chunk=self.chunk, stream=stream)
            sim.load(w)
        return sim, len(w["particles"]["x"])

    def run(self, requests: list[Request]) -> list[Result]:
        torch = self.torch
        pending = sorted(requests, key=lambda r: r.arrival)
        waiting: list[Request] = []
        prepping: dict = {}
        running: dict[int, _Running] = {}
        results: list[Result] = []
        used = 0
        batch = None
        batch_arena = None
        dirty = True
        t0 = time.perf_counter()
        now = lambda: time.perf_counter() - t0
        while pending or waiting or prepping or running:
            t = now()
            while pending and pending[0].arrival <= t:
                waiting.append(pending.pop(0))
            # admission in arrival order while the HBM budget allows
            while waiting:
                r = waiting[0]
                nb = self._bytes(r)
                if used + nb > self.budget and (running or prepping):
                    break
                waiting.pop(0)
                used += nb
                prepping[self.pool.submit(self._prepare, r)] = (r, nb, now())
                self.timeline.append((now(), "admit", r.rid))
            for f in [f for f in prepping if f.done()]:
                r, nb, ta = prepping.pop(f)
                sim, n0 = f.result()
                running[r.rid] = _Running(r, sim, nb, ta, now(), n0)
                self.timeline.append((now(), "start", r.rid))
                dirty = True
            if not running:
                nxt = pending[0].arrival if pending else None
                if prepping:
                    cf.wait(list(prepping), timeout=0.05, return_when=cf.FIRST_COMPLETED)
                elif nxt is not None:
                    time.sleep(max(0.0, min(0.05, nxt - now())))
                continue
            self.max_resident = max(self.max_resident, len(running))
            if dirty:
                if batch is not None:
                    binding.pic_batch_destroy(batch)
                handles = [rr.sim.h for rr in running.values()]
                nbytes = binding.pic_batch_required_bytes(handles)
                batch_arena = torch.empty(nbytes + 256, dtype=torch.uint8, device="cuda")
                ptr = (batch_arena.data_ptr() + 255) // 256 * 256
                batch = binding.pic_batch_create(handles, ptr, nbytes, self.stream.cuda_stream)
                dirty = False
            q = min(self.quantum, min(rr.remaining for rr in running.values()))
            binding.pic_batch_step(batch, q)
            self.stream.synchronize()
            for rid in list(running):
                rr = running[rid]
                rr.remaining -= q
                if rr.remaining == 0:
                    sim = rr.sim
                    sim.sync()
                    e = sim.energy()
                    ax = sim.ex_axis()
                    npart = sim.num_particles()
                    tc = now()
                    results.append(Result(
                        rid=rid, arrival=rr.req.arrival, admitted=rr.admitted, started=rr.started,
                        completed=tc, steps=rr.req.steps,
                        pushes=0.5 * (rr.n_start + npart) * rr.req.steps, energy=e, ex_axis=ax,
                        particles=npart, arena_bytes=rr.nbytes))
                    self.timeline.append((tc, "done", rid))
                    sim.close()
                    del running[rid]
                    used -= rr.nbytes
                    dirty = True
        if batch is not None:
            binding.pic_batch_destroy(batch)
        self.pool.shutdown(wait=True)
        return sorted(results, key=lambda r: r.rid)


def run_alone(r: Request, precision: int = binding.PIC_FP32, chunk: int = 0, patch=(32, 32)):
    """The same request stepped by itself (single-sim graph): energy and axis field."""
    w = request_workload(r, patch)
    sim = binding.Sim(w["params"], precision=precision, capacity=request_capacity(r), chunk=chunk)
    sim.load(w)
    sim.step(r.steps)
    sim.sync()
    out = (sim.energy(), sim.ex_axis(), sim.num_particles())
    sim.close()
    return out


def summarize(results: list[Result]) -> dict:
    lat = np.array([r.completed - r.arrival for r in results])
    wall = max(r.completed for r in results) - min(r.arrival for r in results)
    pushes = sum(r.pushes for r in results)
    return {"requests": len(results), "p50_s": float(np.percentile(lat, 50)),
            "p99_s": float(np.percentile(lat, 99)), "mean_s": float(lat.mean()),
            "wall_s": float(wall), "pushes": float(pushes),
            "aggregate_pushes_per_s": float(pushes / wall) if wall > 0 else math.nan}
