"""Long LWFA runs and the precision sweep: FP32 GPU vs FP64 GPU vs FP64 oracle.

The dynamics are chaotic (bubble formation, injection), so long runs are compared by
diagnostics: total field + kinetic energy at every checkpoint, peak wake amplitude
(|Ex| on axis behind the pulse), relative L2 of Ex on axis (reported), and the
Gauss residual div E - rho_e - rho_ion with the immobile ion lattice of the lab
frame placed in the current window (reported, away from the window's x edges,
where particles leave and enter).
"""
import math

import numpy as np
import pytest

import oracle as orc
from paper_1511_03878_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def binding():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1511_03878_gb300 import binding as b, build

    build.build()
    return b


def ion_density(p, nshift):
    """Charge density of the immobile ions (the electrons' lattice in the lab frame,
    weights n(x_lab) dV/ppc) on the nodes of the current window."""
    nx, ny = p["n"][0], p["n"][1]
    dx, dy = p["d"][0], p["d"][1]
    px, py = p["inject_ppc"][0], p["inject_ppc"][1]
    xs, ys = inputs._lattice_2d(0, nx, ny, dx, dy, (px, py))
    xl = xs + nshift * dx
    dens = p["n0"] * np.clip((xl - p["ramp_x0"]) / p["ramp_len"], 0.0, 1.0)
    keep = dens > 0
    c = orc.make_config(2, p["n"][:2], p["d"][:2], p["dt"], window=True)
    w = dens[keep] * dx * dy / (px * py)
    return orc.rho(c, xs[keep], ys[keep], None, w, +1.0)


class Run:
    """Diagnostics history of one simulation (GPU sim or oracle).

    The paraxial pulse starts with div E != 0 (E_y only); Ampere's law keeps that
    residual fixed in the lab frame, so the conserved quantity is the change of
    div E - rho_e - rho_ion against the initial residual moved by the window shifts."""

    def __init__(self, p, div_minus_rho_e0):
        self.p = p
        self.r0 = div_minus_rho_e0 - ion_density(p, 0)
        self.energy, self.wake, self.axis, self.resid = [], [], [], []

    def record(self, energy, ex_axis, div_minus_rho_e, nshift):
        p = self.p
        self.energy.append(float(np.sum(energy)))
        self.axis.append(ex_axis.copy())
        nx = p["n"][0]
        # behind the pulse: x < x_c - 3 tau (window frame)
        back = int((p["xc"] - 3 * p["tau"]) / p["d"][0])
        self.wake.append(float(np.abs(ex_axis[8:max(back, 9)]).max()))
        r = div_minus_rho_e - ion_density(p, nshift)
        m = 8
        if nshift < nx - 2 * m - 1:
            d = r[:, m:nx - m - nshift] - self.r0[:, m + nshift:nx - m]
            self.resid.append(float(np.abs(d).max()))


def gpu_run(binding, w, prec, steps, every):
    p = w["params"]
    n = len(w["particles"]["x"])
    nfull = p["n"][0] * p["n"][1] * 4
    sim = binding.Sim(p, precision=prec, capacity=3 * nfull + n, chunk=0)
    binding.pic_load_particles(sim.h, w["particles"])
    binding.pic_load_fields(sim.h, w["E"], w["B"], np.zeros(sim.fshape))
    run = Run(p, sim.gauss())
    for _ in range(steps // every):
        sim.step(every)
        _, nshift = sim.step_info()
        run.record(sim.energy(), sim.ex_axis(), sim.gauss(), nshift)
    sim.close()
    return run


def oracle_run(w, steps, every):
    p = w["params"]
    c = orc.make_config(2, p["n"][:2], p["d"][:2], p["dt"], window=True, q=p["q"], m=p["m"],
                        n0=p["n0"], ramp_x0=p["ramp_x0"], ramp_len=p["ramp_len"],
                        inject_ppc=p["inject_ppc"], order=p.get("maxwell_order", 2))
    o = orc.OracleSim(c, 3 * p["n"][0] * p["n"][1] * 4)
    o.set_particles(w["particles"])
    o.set_fields(w["E"], w["B"])
    o.set_rho_bg(np.zeros((p["n"][1], p["n"][0])))
    run = Run(p, o.gauss())
    for _ in range(steps // every):
        o.step(every)
        f = o.get_fields()
        run.record(o.energy(), f["Ex"][p["n"][1] // 2], o.gauss(), o.shifts)
    return run


def rel(a, b, floor=0.0):
    """Relative difference where |b| is above `floor` (zero elsewhere)."""
    a, b = np.asarray(a), np.asarray(b)
    ok = np.abs(b) > floor
    out = np.zeros_like(b, dtype=float)
    out[ok] = np.abs(a[ok] - b[ok]) / np.abs(b[ok])
    return out


def axis_l2(a, b):
    return [float(np.linalg.norm(x - y) / max(np.linalg.norm(y), 1e-30)) for x, y in zip(a, b)]


def test_precision_sweep_reduced_with_oracle(binding):
    """512x128 window (same dx, dy, dt, a0 = 4, 2 particles per cell): 1000 steps,
    FP64 and FP32 GPU vs the FP64 oracle. Gate: energy history and peak wake within 1 %."""
    w = inputs.lwfa2d(nx=512, ny=128, ppc=(2, 1), n0=0.01, ramp_cells=64, a0=4.0, w0=15.0,
                      tau=8.0, laser_back=16.0, patch=(32, 32))
    steps, every = 1000, 100
    o = oracle_run(w, steps, every)
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


def test_precision_sweep_full_size_gpu(binding):
    """2048x512 LWFA (plasma from the pulse centre, 1M particles growing with the
    window), 2000 steps: FP32 vs FP64 on the GPU. Gate: energy history and peak wake
    within 1 %; axis L2 and the Gauss residual are reported."""
    w = inputs.lwfa2d()
    steps, every = 2000, 200
    g64 = gpu_run(binding, w, binding.PIC_FP64, steps, every)
    g32 = gpu_run(binding, w, binding.PIC_FP32, steps, every)
    e = rel(g32.energy, g64.energy)
    k = rel(g32.wake, g64.wake, 0.05 * max(g64.wake))
    print("\nfull sweep (2048x512, 2000 steps), checkpoints every 200 steps")
    print("energy fp64:", np.array2string(np.array(g64.energy), precision=4))
    print("energy rel diff fp32 vs fp64:", np.array2string(e, precision=2))
    print("peak wake fp64:", np.array2string(np.array(g64.wake), precision=4))
    print("peak wake rel fp32 vs fp64:", np.array2string(k, precision=2))
    print("Ex axis L2 rel fp32 vs fp64:",
          np.array2string(np.array(axis_l2(g32.axis, g64.axis)), precision=2))
    print("Gauss residual max  fp64 %.2e  fp32 %.2e" % (max(g64.resid), max(g32.resid)))
    assert e.max() < 0.01
    assert k.max() < 0.01


def test_sixth_order_long_run_with_oracle(binding):
    """The reduced window of the sweep above with the sixth-order solver (dt = 0.76 of
    Yee's limit), 1000 steps: FP64 and FP32 GPU vs the FP64 oracle. Gate: energy history
    and peak wake within 1 %. The Gauss residual is reported only: with this solver
    Esirkepov's current does not keep it at round-off (the two-point divergence)."""
    w = inputs.lwfa2d(nx=512, ny=128, ppc=(2, 1), n0=0.01, ramp_cells=64, a0=4.0, w0=15.0,
                      tau=8.0, laser_back=16.0, patch=(32, 32), cfl=0.76)
    w = dict(w, params=dict(w["params"], maxwell_order=6))
    steps, every = 1000, 100
    o = oracle_run(w, steps, every)
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
