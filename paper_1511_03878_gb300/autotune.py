"""Autotuner for the patch size and the work-queue chunk of a workload.

Both knobs trade the same costs against each other on one GPU:

* a larger patch stages a larger field tile per work item (fewer tile loads and current
  flushes per particle), but needs more shared memory, so fewer CTAs stay resident,
  and gives fewer, coarser items to spread over the 152 SMs;
* a smaller chunk splits a dense patch over more CTAs (the single-GPU form of trading
  patches between processes to even out the load, Sec. 3.1, with the load of a patch
  its particle count, Sec. 3), but every extra item reloads the patch's tile and
  flushes its own current tile.

The best pair depends on the grid, on how particles spread over patches and on the
precision, so it is measured, not modelled. Every candidate is built with the library
(``pic_create``), loaded with the same workload, stepped ``warmup`` times untimed and
``steps`` times timed with CUDA events on its stream; the cost is the time per particle
push. The search is coordinate descent: all patch candidates at the default chunk, then
all chunk candidates at the best patch; a candidate must beat the incumbent by more than
a margin (3 %) to replace it, starting from the workload's own patch. The timed window
(100 steps after 10 warm-up steps by default) has to be long enough to include the
capacity repacks that small patches trigger as the plasma is compressed. Candidates that the library rejects
(``pic_required_bytes`` returns 0: a side that does not divide the grid, or tiles that
do not fit in shared memory) are skipped without touching the GPU.
"""
from __future__ import annotations

import dataclasses
import itertools
import json
import os
import time

from . import binding

PATCH_SIDES = (8, 16, 32, 64)
# layouts measured on a GB300 for the standard workloads, keyed like the in-process cache
TUNING_TABLE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "tuned_layouts.json")
CHUNKS = (512, 1024, 2048, 4096, 8192, 16384)
DEFAULT_CHUNK = 2048


@dataclasses.dataclass
class Choice:
    patch: tuple
    chunk: int
    ns_per_push: float
    # (patch, chunk, ns per push) for every candidate measured, in measuring order
    table: list
    seconds: float


def patch_candidates(params: dict, precision: int, sides=PATCH_SIDES, max_aspect: int = 2):
    """Patch shapes the library accepts for this grid and precision, with side ratios
    at most `max_aspect` (long thin patches stage more guard cells per interior cell)."""
    dims = int(params["dims"])
    out = []
    for p in itertools.product(sides, repeat=dims):
        if max(p) > max_aspect * min(p):
            continue
        cfg = binding.make_config(dict(params, patch=p), precision, capacity=1, chunk=0)
        if binding.pic_required_bytes(cfg) == 0:
            continue
        out.append(tuple(int(v) for v in p))
    return out


def _key(workload: dict, precision: int, patches, chunks) -> str:
    p = workload["params"]
    dims = int(p["dims"])
    extra = {}
    if int(p.get("maxwell_order", 2)) != 2:  # keys of the Yee solver stay as they were
        extra = {"maxwell_order": int(p["maxwell_order"]), "dt": float(p["dt"])}
    return json.dumps({**extra, "dims": dims, "n": list(p["n"][:dims]), "d": list(p["d"][:dims]),
                       "precision": int(precision), "window": bool(p.get("window")),
                       "particles": int(len(workload["particles"]["x"])),
                       "patches": None if patches is None else [list(q) for q in patches],
                       "chunks": [int(c) for c in chunks]})


_CACHE: dict = {}


def measure(workload: dict, precision: int, patch, chunk: int, capacity: int,
            warmup: int = 3, steps: int = 10) -> float:
    """Nanoseconds per particle push of one candidate (CUDA events on the sim's stream)."""
    import torch

    params = dict(workload["params"], patch=tuple(patch))
    sim = binding.Sim(params, precision=precision, capacity=capacity, chunk=chunk)
    try:
        sim.load(workload)
        sim.step(warmup)
        sim.sync()
        n0 = sim.num_particles()
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        ev0.record(sim.stream)
        sim.step(steps)
        ev1.record(sim.stream)
        ev1.synchronize()
        sim.sync()  # raises on any latched device error
        n1 = sim.num_particles()
        ms = ev0.elapsed_time(ev1)
    except binding.PicError as e:
        if e.code not in (binding.PIC_ERR_CAPACITY,):
            raise
        return float("inf")  # this layout overflows its buffers: not a candidate
    finally:
        sim.close()
        del sim
    pushes = steps * 0.5 * (n0 + n1)
    return ms * 1e6 / max(pushes, 1.0)


def _better(r, best, margin):
    """A candidate replaces the incumbent only when it is faster by more than `margin`
    (relative), so run-to-run noise does not move the layout away from the first one
    measured (the workload's own patch at the default chunk)."""
    if best is None or r[2] < (1.0 - margin) * best[2]:
        return r
    return best


def tune(workload: dict, precision: int, capacity: int, patches=None, chunks=CHUNKS,
         warmup: int = 10, steps: int = 100, margin: float = 0.03,
         cache_file: str | None = None) -> Choice:
    """Pick (patch, chunk) for `workload` at `precision` by measurement.

    `capacity` is the particle-slot count each candidate sim gets. Results are cached
    per (grid, cell sizes, precision, window, particle count, candidate lists) in this
    process and, if
    `cache_file` is given, in that JSON file."""
    import torch

    key = _key(workload, precision, patches, chunks)
    if key in _CACHE:
        return _CACHE[key]
    if cache_file and os.path.exists(cache_file):
        with open(cache_file) as f:
            disk = json.load(f)
        if key in disk:
            d = disk[key]
            c = Choice(tuple(d["patch"]), int(d["chunk"]), float(d["ns_per_push"]),
                       [tuple(r) for r in d["table"]], float(d["seconds"]))
            _CACHE[key] = c
            return c
    t0 = time.perf_counter()
    cands = list(patches) if patches is not None else patch_candidates(workload["params"],
                                                                         precision)
    if not cands:
        raise ValueError("no patch candidate fits this grid and precision")
    table = []
    start = tuple(workload["params"].get("patch", cands[0]))
    order = sorted(cands, key=lambda q: tuple(q) != start)  # the given patch first
    best = None
    for p in order:
        r = (tuple(p), DEFAULT_CHUNK,
             measure(workload, precision, p, DEFAULT_CHUNK, capacity, warmup, steps))
        table.append(r)
        best = _better(r, best, margin)
    for c in chunks:
        if c == DEFAULT_CHUNK:
            continue
        r = (best[0], int(c), measure(workload, precision, best[0], c, capacity, warmup, steps))
        table.append(r)
        best = _better(r, best, margin)
    torch.cuda.empty_cache()
    choice = Choice(best[0], best[1], best[2], table, time.perf_counter() - t0)
    _CACHE[key] = choice
    if cache_file:
        disk = {}
        if os.path.exists(cache_file):
            with open(cache_file) as f:
                disk = json.load(f)
        disk[key] = dataclasses.asdict(choice)
        with open(cache_file, "w") as f:
            json.dump(disk, f)
    return choice
