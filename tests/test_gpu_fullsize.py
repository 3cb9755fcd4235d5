"""Parity at the full sizes the bench times, in the launch layouts it can pick.

* LWFA 2048x512 with the window full of plasma (4 194 304 particles, the bench's
  workload), FP64 and double-word: element by element against the oracle after 1 step
  (1e-12) and after 3 steps (1e-9; the window shifts once and injects one column), in
  the default layout and at both ends of the autotuner's patch/chunk range.
* 3D stress 256x128x128 with 64M particles over 8^3 patches: the oracle would need
  minutes per step here, so the full size is checked through properties that hold at
  any size, with expected values computed from the inputs alone:
  - from zero fields, the first push leaves every momentum unchanged, so the current of
    step 1 must satisfy sum_cells J dV = sum_p q w u/gamma (Esirkepov's deposit moves
    each particle's charge exactly along its path);
  - the change of div E - rho stays at round-off (FP64) or at the stated FP32 level;
  - the particle count is conserved (periodic box).
"""
import numpy as np
import pytest

import oracle as orc
from paper_1511_03878_gb300 import inputs

pytestmark = pytest.mark.gpu

FIELD_KEYS = ("Ex", "Ey", "Ez", "Bx", "By", "Bz", "Bnx", "Bny", "Bnz", "Jx", "Jy", "Jz")


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
    if den == 0:
        return float(np.abs(a).max())
    return float(np.abs(a - b).max() / den)


@pytest.fixture(scope="module")
def lwfa_full():
    """The bench's LWFA window and the oracle's state after 1 and after 3 steps."""
    w = inputs.lwfa2d(nx=2048, ny=512, ramp_x0=-8.0)
    p = w["params"]
    c = orc.make_config(2, p["n"][:2], p["d"][:2], p["dt"], window=True, q=p["q"], m=p["m"],
                        n0=p["n0"], ramp_x0=p["ramp_x0"], ramp_len=p["ramp_len"],
                        inject_ppc=p["inject_ppc"])
    n = len(w["particles"]["x"])
    o = orc.OracleSim(c, n + 100000)
    o.set_particles(w["particles"])
    o.set_fields(w["E"], w["B"])
    o.set_rho_bg(None)
    snaps = {}
    for k, upto in ((1, 1), (3, 2)):
        o.step(upto)
        snaps[k] = (o.get_fields(), o.get_particles(), o.shifts)
    return w, snaps


def compare_snapshot(sim, snap, params, tol, tol_j=None):
    fo, qo, shifts = snap
    f = sim.fields()
    errs = {k: normwise(f[k], fo[k]) for k in FIELD_KEYS}
    q = sim.particles()
    assert np.array_equal(q["id"], qo["id"])
    Ly = params["n"][1] * params["d"][1]
    dy = (q["y"] - qo["y"] + 0.5 * Ly) % Ly - 0.5 * Ly
    errs["x"] = normwise(q["x"], qo["x"])
    errs["y"] = float(np.abs(dy).max() / np.abs(qo["y"]).max())
    for k in ("ux", "uy", "uz", "w"):
        errs[k] = normwise(q[k], qo[k])
    assert sim.step_info()[1] == shifts
    lim = {k: (tol_j if tol_j is not None and k in ("Jx", "Jy", "Jz", "Ex", "Ey", "Ez")
               else tol) for k in errs}
    bad = {k: v for k, v in errs.items() if not v <= lim[k]}
    assert not bad, (bad, errs)
    return errs


@pytest.mark.parametrize("prec", ["fp64", "df64"])
@pytest.mark.parametrize("patch,chunk", [((32, 32), 0), ((64, 32), 512), ((16, 16), 8192)])
def test_lwfa_full_window(binding, lwfa_full, prec, patch, chunk):
    w, snaps = lwfa_full
    P = {"fp64": binding.PIC_FP64, "df64": binding.PIC_DF64}[prec]
    n = len(w["particles"]["x"])
    params = dict(w["params"], patch=patch)
    sim = binding.Sim(params, precision=P, capacity=3 * n, chunk=chunk)
    sim.load(w)
    sim.step(1)
    # Double-word positions keep the in-cell offset to ~2^-48 cells; the oracle keeps FP64
    # positions in global cell units, rounded to ulp(2048)/2 = 2.3e-13 cells at the far
    # end of the window. In the nearly static plasma ahead of the pulse that rounding
    # gives ~1e-15 of current where the current is ~1e-17, i.e. 1.1e-12 of max|Jx|, which
    # the double-word path does not reproduce (the FP64 GPU path shares the oracle's
    # representation and agrees to 3.5e-13). Its current, and E through it, are held to
    # 3e-12 after one step; everything else to 1e-12.
    e1 = compare_snapshot(sim, snaps[1], params, 1e-12, 3e-12 if prec == "df64" else None)
    sim.step(2)
    e3 = compare_snapshot(sim, snaps[3], params, 1e-9)
    print(f"\nLWFA 2048x512 {prec} patch {patch} chunk {chunk}: 1 step max "
          f"{max(e1.values()):.1e}, 3 steps max {max(e3.values()):.1e}")
    sim.close()


@pytest.fixture(scope="module")
def stress_full():
    w = inputs.stress3d()
    w["params"] = dict(w["params"], patch=(8, 8, 8))
    q = w["particles"]
    p = w["params"]
    ig = 1.0 / np.sqrt(1.0 + q["ux"] ** 2 + q["uy"] ** 2 + q["uz"] ** 2)
    qw = p["q"] * q["w"]
    expect = np.array([np.sum(qw * q[k] * ig) for k in ("ux", "uy", "uz")])
    scale = np.array([np.sum(np.abs(qw * q[k] * ig)) for k in ("ux", "uy", "uz")])
    c = orc.make_config(3, p["n"], p["d"], p["dt"], q=p["q"], m=p["m"])
    rho_max = float(np.abs(orc.rho(c, q["x"], q["y"], q["z"], q["w"], p["q"])).max())
    return w, expect, scale, rho_max


# FP32 accumulates each work item's current in an int32 fixed-point tile whose quantum is
# 2^(lg(items) - 30) of the bound on one contribution (items of 8192 particles here):
# the current sum stays at ~4e-8 and the Gauss-law drift at ~1.3e-6 of max rho (it was
# 6e-9 with an FP32 float tile, 2.1x slower)
@pytest.mark.parametrize("prec,tol_j,tol_g", [("fp64", 1e-12, 1e-12), ("fp32", 1e-7, 5e-6)])
def test_stress3d_full_size_invariants(binding, stress_full, prec, tol_j, tol_g):
    w, expect, scale, rho_max = stress_full
    P = {"fp64": binding.PIC_FP64, "fp32": binding.PIC_FP32}[prec]
    n = len(w["particles"]["x"])
    p = w["params"]
    sim = binding.Sim(p, precision=P, capacity=2 * n)
    sim.load(w)
    g0 = sim.gauss()
    sim.step(1)
    f = sim.fields()
    dv = p["d"][0] * p["d"][1] * p["d"][2]
    got = np.array([f[k].sum() * dv for k in ("Jx", "Jy", "Jz")])
    jerr = np.abs(got - expect) / scale
    del f
    sim.step(1)
    gerr = float(np.abs(sim.gauss() - g0).max() / rho_max)
    assert sim.num_particles() == n
    print(f"\n3D stress 64M {prec}: sum J dV vs sum q w v {jerr.max():.1e}, "
          f"Gauss change / max rho {gerr:.1e}")
    assert jerr.max() < tol_j, jerr
    assert gerr < tol_g
    sim.close()
