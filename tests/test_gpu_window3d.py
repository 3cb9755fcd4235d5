"""3D LWFA in a moving window (shift folded into the Yee write index and the particle
store, cold-lattice injection of an ny x nz column) against the oracle."""
import numpy as np
import pytest

import oracle as orc
from paper_1511_03878_gb300 import inputs

pytestmark = pytest.mark.gpu

KEYS = ("Ex", "Ey", "Ez", "Bx", "By", "Bz", "Bnx", "Bny", "Bnz", "Jx", "Jy", "Jz")


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


def small_lwfa3d():
    # plasma from 6 cells behind the pulse centre, pulse 6 units from the right edge
    w = inputs.lwfa3d(nx=64, ny=16, nz=16, ppc=(2, 1, 1), laser_back=6.0, w0=3.0, tau=3.0,
                      ramp_cells=8, patch=(16, 8, 8))
    return inputs.lwfa3d(nx=64, ny=16, nz=16, ppc=(2, 1, 1), laser_back=6.0, w0=3.0, tau=3.0,
                         ramp_cells=8, patch=(16, 8, 8), ramp_x0=w["params"]["xc"] - 6.0)


def oracle_after(w, steps):
    p = w["params"]
    c = orc.make_config(3, p["n"], p["d"], p["dt"], window=True, q=p["q"], m=p["m"], n0=p["n0"],
                        ramp_x0=p["ramp_x0"], ramp_len=p["ramp_len"], inject_ppc=p["inject_ppc"])
    o = orc.OracleSim(c, len(w["particles"]["x"]) + 100000)
    o.set_particles(w["particles"])
    o.set_fields(w["E"], w["B"])
    o.set_rho_bg(None)
    o.step(steps)
    return c, o


@pytest.mark.parametrize("prec", ["fp64"])  # the double-word precision is 2D only
@pytest.mark.parametrize("steps,tol", [(1, 1e-12), (12, 1e-9)])
def test_lwfa3d_window_matches_oracle(binding, prec, steps, tol):
    w = small_lwfa3d()
    P = {"fp64": binding.PIC_FP64, "df64": binding.PIC_DF64}[prec]
    n = len(w["particles"]["x"])
    sim = binding.Sim(w["params"], precision=P, capacity=4 * n + 100000)
    sim.load(w)
    sim.step(steps)
    c, o = oracle_after(w, steps)
    s, k = sim.step_info()
    assert s == steps and k == o.shifts == orc.shift_count(c, steps)
    f, fo = sim.fields(), o.get_fields()
    errs = {key: normwise(f[key], fo[key]) for key in KEYS}
    q, qo = sim.particles(), o.get_particles()
    assert np.array_equal(q["id"], qo["id"])
    p = w["params"]
    for a, key in enumerate(("x", "y", "z")):
        L = p["n"][a] * p["d"][a]
        dd = q[key] - qo[key]
        if a > 0:
            dd = (dd + 0.5 * L) % L - 0.5 * L
        errs[key] = float(np.abs(dd).max() / np.abs(qo[key]).max())
    for key in ("ux", "uy", "uz", "w"):
        errs[key] = normwise(q[key], qo[key])
    bad = {key: v for key, v in errs.items() if not v <= tol}
    assert not bad, (bad, errs)
    assert steps == 1 or k > 0  # the window moved and injected
    sim.close()


def test_lwfa3d_window_fp32_error_stated(binding):
    w = small_lwfa3d()
    n = len(w["particles"]["x"])
    sim = binding.Sim(w["params"], precision=binding.PIC_FP32, capacity=4 * n + 100000)
    sim.load(w)
    sim.step(12)
    c, o = oracle_after(w, 12)
    assert sim.num_particles() == o.num_particles()
    f, fo = sim.fields(), o.get_fields()
    ey = normwise(f["Ey"], fo["Ey"])
    e, eo = sim.energy(), o.energy()
    print(f"FP32 3D window 12 steps: Ey {ey:.2e}, energy {abs(e.sum() / eo.sum() - 1):.2e}")
    assert ey < 1e-4 and abs(e.sum() - eo.sum()) / eo.sum() < 1e-3
    sim.close()
