"""Diagnostics of long LWFA runs, shared by the GPU long-run tests and the script that
writes the oracle's stored long-run diagnostics (tests/golden/make_sweep_golden.py).

The dynamics are chaotic (bubble formation, injection), so long runs are compared by
diagnostics: total field + kinetic energy at every checkpoint, peak wake amplitude
(|Ex| on axis behind the pulse), relative L2 of Ex on axis (reported), and the
Gauss residual div E - rho_e - rho_ion with the immobile ion lattice of the lab
frame placed in the current window (reported, away from the window's x edges,
where particles leave and enter).
"""
import numpy as np

import oracle as orc
from paper_1511_03878_gb300 import inputs


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
        self.energy, self.wake, self.axis, self.resid, self.count = [], [], [], [], []

    def record(self, energy, ex_axis, div_minus_rho_e, nshift, count=None):
        p = self.p
        self.energy.append(float(np.sum(energy)))
        self.axis.append(np.asarray(ex_axis, dtype=np.float64).copy())
        nx = p["n"][0]
        # behind the pulse: x < x_c - 3 tau (window frame)
        back = int((p["xc"] - 3 * p["tau"]) / p["d"][0])
        self.wake.append(float(np.abs(ex_axis[8:max(back, 9)]).max()))
        r = div_minus_rho_e - ion_density(p, nshift)
        m = 8
        if nshift < nx - 2 * m - 1:
            d = r[:, m:nx - m - nshift] - self.r0[:, m + nshift:nx - m]
            self.resid.append(float(np.abs(d).max()))
        if count is not None:
            self.count.append(int(count))


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
        run.record(sim.energy(), sim.ex_axis(), sim.gauss(), nshift, sim.num_particles())
    sim.close()
    return run


def oracle_run(w, steps, every, threads=1):
    """The FP64 oracle over `steps` steps; threads > 1 uses its threaded step, whose
    results are identical bit for bit."""
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
        o.step(every, threads=threads)
        f = o.get_fields()
        run.record(o.energy(), f["Ex"][p["n"][1] // 2], o.gauss(), o.shifts, o.num_particles())
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
