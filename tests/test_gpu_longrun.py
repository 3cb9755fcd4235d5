"""Long LWFA runs and the precision sweep: FP32 GPU vs FP64 GPU vs FP64 oracle.

The dynamics are chaotic (bubble formation, injection), so long runs are compared by
diagnostics (tests/longrun_diag.py): total field + kinetic energy at every checkpoint,
peak wake amplitude (|Ex| on axis behind the pulse), relative L2 of Ex on axis
(reported), and the Gauss residual (reported).
"""
import json
import os

import numpy as np
import pytest

from longrun_diag import axis_l2, gpu_run, oracle_run, rel
from paper_1511_03878_gb300 import inputs

pytestmark = pytest.mark.gpu

# host threads of the oracle's threaded step (results identical bit for bit)
THREADS = os.cpu_count() or 1


@pytest.fixture(scope="module")
def binding():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1511_03878_gb300 import binding as b, build

    build.build()
    return b


def test_precision_sweep_reduced_with_oracle(binding):
    """512x128 window (same dx, dy, dt, a0 = 4, 2 particles per cell): 1000 steps,
    FP64 and FP32 GPU vs the FP64 oracle. Gate: energy history and peak wake within 1 %."""
    w = inputs.lwfa2d(nx=512, ny=128, ppc=(2, 1), n0=0.01, ramp_cells=64, a0=4.0, w0=15.0,
                      tau=8.0, laser_back=16.0, patch=(32, 32))
    steps, every = 1000, 100
    o = oracle_run(w, steps, every, threads=THREADS)
    g64 = gpu_run(binding, w, binding.PIC_FP64, steps, every)
    g32 = gpu_run(binding, w, binding.PIC_FP32, steps, every)
    e64, e32 = rel(g64.energy, o.energy), rel(g32.energy, o.energy)
    wfloor = 0.05 * max(o.wake)  # compare once the wake has formed
    k64, k32 = rel(g64.wake, o.wake, wfloor), rel(g32.wake, o.wake, wfloor)
    print("\nreduced sweep (512x128, 1000 steps), checkpoints every 100 steps")
    print("energy rel diff  fp64:", np.array2string(e64, precision=2))
    print("energy rel diff  fp32:", np.array2string(e32, precision=2))
    print("peak wake (oracle):", np.array2string(np.array(o.wake), precision=4))
    print("peak wake rel    fp64:", np.array2string(k64, precision=2))
    print("peak wake rel    fp32:", np.array2string(k32, precision=2))
    print("Ex axis L2 rel   fp64:", np.array2string(np.array(axis_l2(g64.axis, o.axis)), precision=2))
    print("Ex axis L2 rel   fp32:", np.array2string(np.array(axis_l2(g32.axis, o.axis)), precision=2))
    print("Gauss residual max   oracle %.2e  fp64 %.2e  fp32 %.2e" % (
        max(o.resid), max(g64.resid), max(g32.resid)))
    assert e64.max() < 0.01 and e32.max() < 0.01
    assert k64.max() < 0.01 and k32.max() < 0.01


GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "lwfa2048_sweep_oracle.json")


def test_precision_sweep_full_size_vs_oracle(binding):
    """The sweep at its stated size: 2048x512 LWFA (plasma from the pulse centre, 1M
    particles growing with the window to 4.2M), 2000 steps, FP64 and FP32 on the GPU
    against the FP64 oracle's diagnostics of the same run, stored by
    tests/golden/make_sweep_golden.py (oracle only). Gate: energy history and peak
    wake within 1 % at every checkpoint (every 100 steps); Ex-axis L2, the Gauss
    residual and the particle count are reported."""
    with open(GOLDEN) as f:
        ref = json.load(f)
    w = inputs.lwfa2d()
    steps, every = ref["steps"][-1], ref["steps"][0]
    g64 = gpu_run(binding, w, binding.PIC_FP64, steps, every)
    g32 = gpu_run(binding, w, binding.PIC_FP32, steps, every)
    wfloor = 0.05 * max(ref["wake"])
    print("\nfull sweep vs oracle (2048x512, %d steps), checkpoints every %d" % (steps, every))
    print("energy (oracle):", np.array2string(np.array(ref["energy"]), precision=5))
    print("peak wake (oracle):", np.array2string(np.array(ref["wake"]), precision=4))
    out = {}
    for name, g in (("fp64", g64), ("fp32", g32)):
        e = rel(g.energy, ref["energy"])
        k = rel(g.wake, ref["wake"], wfloor)
        ax = {s: axis_l2([g.axis[ref["steps"].index(int(s))]], [np.array(v)])[0]
              for s, v in ref["axis"].items()}
        out[name] = (e, k)
        print("%s energy rel diff:" % name, np.array2string(e, precision=2))
        print("%s peak wake rel:  " % name, np.array2string(k, precision=2))
        print("%s Ex axis L2 rel at steps %s: %s" % (
            name, list(ax), ", ".join("%.2e" % v for v in ax.values())))
        print("%s Gauss residual max %.2e (oracle %.2e); particles %d (oracle %d)" % (
            name, max(g.resid), max(ref["resid"]), g.count[-1], ref["count"][-1]))
    for name, (e, k) in out.items():
        assert e.max() < 0.01, (name, e.max())
        assert k.max() < 0.01, (name, k.max())
    # FP64 reproduces the oracle's run far inside the 1 % gate (measured on a GB300:
    # energy 7e-13, peak wake 1e-11, axis L2 1e-10 after 2000 steps): a regression guard
    # four orders of magnitude above that
    e64, k64 = out["fp64"]
    assert e64.max() < 1e-6 and k64.max() < 1e-6, (e64.max(), k64.max())
    # charge conservation in FP32 (int32 fixed-point current tile): the change of
    # div E - rho stays at 2.8e-5 (measured; the oracle's is 2.4e-14) against charge
    # densities of about 0.01 to 0.1
    assert max(g32.resid) < 1e-4, max(g32.resid)
    assert abs(g64.count[-1] - ref["count"][-1]) <= 2  # particles leaving at the window edge


def test_sixth_order_long_run_with_oracle(binding):
    """The reduced window of the sweep above with the sixth-order solver (dt = 0.76 of
    Yee's limit), 1000 steps: FP64 and FP32 GPU vs the FP64 oracle. Gate: energy history
    and peak wake within 1 %. The Gauss residual is reported only: with this solver
    Esirkepov's current does not keep it at round-off (the two-point divergence)."""
    w = inputs.lwfa2d(nx=512, ny=128, ppc=(2, 1), n0=0.01, ramp_cells=64, a0=4.0, w0=15.0,
                      tau=8.0, laser_back=16.0, patch=(32, 32), cfl=0.76)
    w = dict(w, params=dict(w["params"], maxwell_order=6))
    steps, every = 1000, 100
    o = oracle_run(w, steps, every, threads=THREADS)
    g64 = gpu_run(binding, w, binding.PIC_FP64, steps, every)
    g32 = gpu_run(binding, w, binding.PIC_FP32, steps, every)
    e64, e32 = rel(g64.energy, o.energy), rel(g32.energy, o.energy)
    wfloor = 0.05 * max(o.wake)
    k64, k32 = rel(g64.wake, o.wake, wfloor), rel(g32.wake, o.wake, wfloor)
    print("\nsixth-order solver, reduced window (512x128, 1000 steps)")
    print("energy rel diff  fp64:", np.array2string(e64, precision=2))
    print("energy rel diff  fp32:", np.array2string(e32, precision=2))
    print("peak wake rel    fp64:", np.array2string(k64, precision=2))
    print("peak wake rel    fp32:", np.array2string(k32, precision=2))
    print("Ex axis L2 rel   fp64:", np.array2string(np.array(axis_l2(g64.axis, o.axis)), precision=2))
    print("Gauss residual max   oracle %.2e  fp64 %.2e  fp32 %.2e" % (
        max(o.resid), max(g64.resid), max(g32.resid)))
    assert e64.max() < 0.01 and e32.max() < 0.01
    assert k64.max() < 0.01 and k32.max() < 0.01
