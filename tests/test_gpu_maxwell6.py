"""Sixth-order Maxwell solver (Sec. 2.1's higher-order scheme) on the GPU against the
oracle, element by element, with the tolerances of the Yee tests: FP64 and double-word
1e-12 after one step and 1e-9 after up to 20 steps; FP32 with its error stated.

Covered: 2D periodic (thermal plasma), 2D moving window with injection (the wide
stencil reads the column each shift drops), 3D periodic and 3D window, and the host
check that a batch does not mix solver orders. The time steps are 0.76 of Yee's limit,
below the sixth-order limit 120/149 = 0.805 of it.
"""
import numpy as np
import pytest

import oracle as orc
from paper_1511_03878_gb300 import inputs

pytestmark = pytest.mark.gpu

KEYS = ("Ex", "Ey", "Ez", "Bx", "By", "Bz", "Bnx", "Bny", "Bnz", "Jx", "Jy", "Jz")
CFL6 = 0.76
PREC64 = {"fp64": 0, "df64": 2}


@pytest.fixture(scope="module")
def binding():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1511_03878_gb300 import binding as b, build

    build.build()
    return b


def normwise(a, b):
    den = np.abs(b).max()
    return float(np.abs(a - b).max() / den) if den > 0 else float(np.abs(a).max())


def sixth(w):
    return dict(w, params=dict(w["params"], maxwell_order=6))


def oracle_after(w, steps):
    p = w["params"]
    dims = p["dims"]
    c = orc.make_config(dims, p["n"][:dims], p["d"][:dims], p["dt"], window=p["window"],
                        q=p["q"], m=p["m"], n0=p["n0"], ramp_x0=p["ramp_x0"],
                        ramp_len=p["ramp_len"], inject_ppc=p["inject_ppc"],
                        order=p.get("maxwell_order", 2))
    o = orc.OracleSim(c, 4 * len(w["particles"]["x"]) + 100000)
    o.set_particles(w["particles"])
    o.set_fields(w["E"], w["B"])
    o.set_rho_bg(None)
    o.step(steps)
    return c, o


def errors(sim, o, params):
    f, fo = sim.fields(), o.get_fields()
    errs = {k: normwise(f[k], fo[k]) for k in KEYS}
    q, qo = sim.particles(), o.get_particles()
    assert np.array_equal(q["id"], qo["id"])
    dims = params["dims"]
    for a, key in enumerate(("x", "y", "z")[:dims]):
        L = params["n"][a] * params["d"][a]
        dd = q[key] - qo[key]
        if a > 0 or not params["window"]:
            dd = (dd + 0.5 * L) % L - 0.5 * L
        errs[key] = float(np.abs(dd).max() / np.abs(qo[key]).max())
    for key in ("ux", "uy", "uz", "w"):
        errs[key] = normwise(q[key], qo[key])
    return errs


def run_and_compare(binding, w, prec, steps, tol, capacity):
    sim = binding.Sim(w["params"], precision=prec, capacity=capacity)
    sim.load(w)
    sim.step(steps)
    c, o = oracle_after(w, steps)
    s, k = sim.step_info()
    assert s == steps and k == o.shifts
    errs = errors(sim, o, w["params"])
    sim.close()
    return errs, k


def small_lwfa():
    args = dict(nx=256, ny=128, dx=0.125, dy=0.5, ppc=(2, 2), n0=0.01, ramp_cells=16,
                a0=4.0, w0=15.0, tau=8.0, laser_back=12.0, patch=(32, 32), cfl=CFL6)
    w = inputs.lwfa2d(**args)
    return sixth(inputs.lwfa2d(**args, ramp_x0=w["params"]["xc"] - 8.0))


def small_lwfa3d():
    args = dict(nx=64, ny=16, nz=16, ppc=(2, 1, 1), laser_back=6.0, w0=3.0, tau=3.0,
                ramp_cells=8, patch=(16, 8, 8), cfl=CFL6)
    w = inputs.lwfa3d(**args)
    return sixth(inputs.lwfa3d(**args, ramp_x0=w["params"]["xc"] - 6.0))


@pytest.mark.parametrize("prec", ["fp64", "df64"])
@pytest.mark.parametrize("steps,tol", [(1, 1e-12), (20, 1e-9)])
def test_thermal_2d_periodic(binding, prec, steps, tol):
    w = sixth(inputs.thermal2d(seed=1511, cfl=CFL6))
    n = len(w["particles"]["x"])
    errs, _ = run_and_compare(binding, w, PREC64[prec], steps, tol, 2 * n)
    bad = {k: v for k, v in errs.items() if not v <= tol}
    assert not bad, (bad, errs)


@pytest.mark.parametrize("prec", ["fp64", "df64"])
@pytest.mark.parametrize("steps,tol", [(1, 1e-12), (20, 1e-9)])
def test_lwfa_2d_window(binding, prec, steps, tol):
    w = small_lwfa()
    n = len(w["particles"]["x"])
    errs, shifts = run_and_compare(binding, w, PREC64[prec], steps, tol, 8 * n + 100000)
    bad = {k: v for k, v in errs.items() if not v <= tol}
    assert not bad, (bad, errs)
    assert steps == 1 or shifts >= 10


@pytest.mark.parametrize("prec", ["fp64"])  # the double-word precision is 2D only
@pytest.mark.parametrize("steps,tol", [(1, 1e-12), (12, 1e-9)])
def test_3d_periodic(binding, prec, steps, tol):
    w = sixth(inputs.stress3d(n=(32, 16, 16), patch=(8, 8, 8), total=60000, cfl=CFL6))
    n = len(w["particles"]["x"])
    errs, _ = run_and_compare(binding, w, PREC64[prec], steps, tol, 4 * n)
    bad = {k: v for k, v in errs.items() if not v <= tol}
    assert not bad, (bad, errs)


@pytest.mark.parametrize("prec", ["fp64"])  # the double-word precision is 2D only
@pytest.mark.parametrize("steps,tol", [(1, 1e-12), (12, 1e-9)])
def test_3d_window(binding, prec, steps, tol):
    w = small_lwfa3d()
    n = len(w["particles"]["x"])
    errs, shifts = run_and_compare(binding, w, PREC64[prec], steps, tol, 4 * n + 100000)
    bad = {k: v for k, v in errs.items() if not v <= tol}
    assert not bad, (bad, errs)
    assert steps == 1 or shifts >= 6


def test_fp32_window_error_stated(binding):
    """FP32 particles and fields (FP64 current) after 20 steps in the 2D window:
    momenta and positions within 1e-4 of the FP64 oracle, the laser field Ey within
    1e-4, the field energy within 1e-3 (the Yee FP32 test's bounds)."""
    w = small_lwfa()
    n = len(w["particles"]["x"])
    sim = binding.Sim(w["params"], precision=binding.PIC_FP32, capacity=8 * n + 100000)
    sim.load(w)
    sim.step(20)
    _, o = oracle_after(w, 20)
    errs = errors(sim, o, w["params"])
    e, eo = sim.energy(), np.array(o.energy())
    sim.close()
    assert errs["ux"] < 1e-4 and errs["x"] < 1e-4 and errs["Ey"] < 1e-4, errs
    assert abs(e.sum() - eo.sum()) / eo.sum() < 1e-3


def test_batch_refuses_mixed_solver_orders(binding):
    w2 = inputs.thermal2d(nx=64, ny=64, patch=(16, 16), cfl=CFL6)
    w6 = sixth(w2)
    n = len(w2["particles"]["x"])
    a = binding.Sim(w2["params"], precision=binding.PIC_FP64, capacity=2 * n)
    b = binding.Sim(w6["params"], precision=binding.PIC_FP64, capacity=2 * n)
    c = binding.Sim(w6["params"], precision=binding.PIC_FP64, capacity=2 * n)
    try:
        assert binding.pic_batch_required_bytes([a.h, b.h]) == 0
        assert binding.pic_batch_required_bytes([b.h, c.h]) > 0
    finally:
        for s in (a, b, c):
            s.close()


def _group_velocity(order, k, dx, dt):
    """dω/dk of the 1D discrete vacuum relation sin(ω dt/2) = (dt/2) K(k), where K is the
    symbol of the staggered difference (Yee: (2/dx) sin(k dx/2); sixth order: the c_l sum)."""
    c = (1.0,) if order == 2 else (75 / 64, -25 / 384, 3 / 640)

    def omega(kk):
        K = 2 / dx * sum(cl * np.sin((2 * l + 1) * kk * dx / 2) for l, cl in enumerate(c))
        return 2 / dt * np.arcsin(dt * K / 2)

    h = 1e-4
    return (omega(k + h) - omega(k - h)) / (2 * h)


@pytest.mark.parametrize("order,cfl", [(2, 0.95), (6, 0.76)])
def test_laser_group_velocity_in_vacuum(binding, order, cfl):
    """Sec. 2.1: the second-order scheme propagates a laser pulse slower than light and
    the sixth-order one faster. A pulse uniform in y (no diffraction) crosses a vacuum
    moving window in FP64; the lab-frame drift of its energy centroid gives the group
    velocity, which must match the discrete dispersion relation at k0 = 1 within 10 %
    of its offset from c and have the predicted sign."""
    w = inputs.lwfa2d(nx=512, ny=32, n0=0.0, laser_back=24.0, tau=8.0, patch=(32, 32), cfl=cfl)
    p = dict(w["params"], maxwell_order=order)
    nx, ny = p["n"][0], p["n"][1]
    dx, dt, xc = p["d"][0], p["dt"], p["xc"]
    x = np.arange(nx) * dx
    env = lambda s: np.exp(-2.0 * np.log(2.0) * (s - xc) ** 2 / 8.0 ** 2) * np.cos(s - xc)
    E = [np.zeros((ny, nx)), np.repeat(env(x)[None, :], ny, 0), np.zeros((ny, nx))]
    B = [np.zeros((ny, nx)), np.zeros((ny, nx)), np.repeat(env(x + 0.5 * dx - 0.5 * dt)[None, :], ny, 0)]
    w = dict(w, params=p, E=E, B=B)
    sim = binding.Sim(p, precision=binding.PIC_FP64, capacity=100000)
    sim.load(w)

    def centroid():
        f = sim.fields()
        ey2 = (f["Ey"] ** 2).sum(axis=0)
        bz2 = (f["Bnz"] ** 2).sum(axis=0)
        xs = (np.sum(x * ey2) + np.sum((x + 0.5 * dx) * bz2)) / (ey2.sum() + bz2.sum())
        return xs + sim.step_info()[1] * dx  # window frame -> lab frame

    n0, n1 = 20, int(round(46.0 / dt))
    sim.step(n0)
    x0 = centroid()
    sim.step(n1 - n0)
    x1 = centroid()
    sim.close()
    vg = (x1 - x0) / ((n1 - n0) * dt)
    want = _group_velocity(order, 1.0, dx, dt)
    print(f"\norder {order}: measured v_g - 1 = {vg - 1:.3e}, dispersion relation {want - 1:.3e}")
    assert np.sign(vg - 1) == np.sign(want - 1) == (-1 if order == 2 else 1)
    assert abs((vg - 1) - (want - 1)) < 0.1 * abs(want - 1)
