"""Writes tests/golden/lwfa2048_sweep_oracle.json: the FP64 oracle's diagnostics of the
full precision-sweep configuration, the 2048x512 LWFA window (dx = 0.125, dy = 0.5,
dt = 0.95 CFL, n0 = 0.01 n_c with a 64-cell ramp from the pulse centre, 4 particles per
cell, a0 = 4, w0 = 30, tau = 25) over 2000 steps, every 100 steps: total energy, peak
wake |Ex| on axis behind the pulse, the Gauss-residual change, the particle count, and
Ex on the axis at steps 1000 and 2000.

It calls only the oracle (its threaded step, identical bit for bit to the plain one)
and the seeded input generator. Run from the repository root:
    python tests/golden/make_sweep_golden.py [threads]
"""
import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)
sys.path.insert(0, os.path.dirname(HERE))

from longrun_diag import oracle_run  # noqa: E402
from paper_1511_03878_gb300 import inputs  # noqa: E402

STEPS, EVERY = 2000, 100
AXIS_AT = (1000, 2000)


def main():
    threads = int(sys.argv[1]) if len(sys.argv) > 1 else (os.cpu_count() or 1)
    w = inputs.lwfa2d()
    t0 = time.time()
    run = oracle_run(w, STEPS, EVERY, threads=threads)
    steps = [EVERY * (k + 1) for k in range(STEPS // EVERY)]
    out = dict(
        config="lwfa2d-2048x512-ppc4, inputs.lwfa2d() defaults (seed 1512), FP64 oracle",
        steps=steps, energy=run.energy, wake=run.wake, resid=run.resid, count=run.count,
        axis={str(s): [float("%.12g" % v) for v in run.axis[steps.index(s)]] for s in AXIS_AT},
        threads=threads, seconds=round(time.time() - t0, 1))
    with open(os.path.join(HERE, "lwfa2048_sweep_oracle.json"), "w") as f:
        json.dump(out, f, indent=0)
    print("wrote lwfa2048_sweep_oracle.json in %.0f s" % (time.time() - t0))


if __name__ == "__main__":
    main()
