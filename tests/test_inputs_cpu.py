"""The seeded synthetic workloads match the recipe stated for them: grid, time step,
particle counts per cell, momentum spread, weights of the density ramp, the laser's
peak field and the log-normal spread of the 3D stress counts. The generators draw
lattices, momenta and laser fields only; no step of the method is in them."""
import math

import numpy as np

from paper_1511_03878_gb300 import inputs


def test_thermal_plasma():
    w = inputs.thermal2d()
    p, q = w["params"], w["particles"]
    assert tuple(p["n"][:2]) == (128, 128) and tuple(p["d"][:2]) == (0.1, 0.1)
    assert abs(p["dt"] - 0.95 / math.sqrt(2.0 / 0.01)) < 1e-12
    assert len(q["x"]) == 262_144
    counts = np.histogram2d(q["x"], q["y"], bins=128, range=[[0, 12.8], [0, 12.8]])[0]
    assert (counts == 16).all()  # a 4x4 lattice in every cell
    for k in ("ux", "uy", "uz"):
        assert abs(q[k].std() / 0.044 - 1.0) < 0.01 and abs(q[k].mean()) < 5e-4
    assert abs(q["w"].sum() - 12.8 * 12.8) < 1e-9  # density 1
    assert np.unique(q["id"]).size == q["id"].size
    assert not any(np.abs(a).max() for a in w["E"] + w["B"])


def test_lwfa_window():
    w = inputs.lwfa2d()
    p, q = w["params"], w["particles"]
    dx, dy = p["d"][0], p["d"][1]
    assert tuple(p["n"][:2]) == (2048, 512) and (dx, dy) == (0.125, 0.5)
    assert abs(p["dt"] - 0.95 / math.sqrt(1 / dx ** 2 + 1 / dy ** 2)) < 1e-12
    # plasma from the laser centre on, a 64-cell ramp, 2x2 per cell, cold
    assert p["ramp_x0"] == p["xc"] and p["ramp_len"] == 64 * dx and p["n0"] == 0.01
    assert len(q["x"]) == (2048 - int(p["xc"] / dx)) * 512 * 4 == 1_048_576
    assert q["x"].min() > p["ramp_x0"]
    assert not (np.abs(q["ux"]).max() or np.abs(q["uy"]).max() or np.abs(q["uz"]).max())
    plateau = 0.01 * dx * dy / 4
    ramp = np.clip((q["x"] - p["ramp_x0"]) / p["ramp_len"], 0.0, 1.0)
    assert np.allclose(q["w"], plateau * ramp, rtol=1e-12, atol=0)
    # the laser: a0 = 4 at the centre (Ey and Bz sampled on their staggered nodes)
    assert 3.99 < np.abs(w["E"][1]).max() <= 4.0 and 3.99 < np.abs(w["B"][2]).max() <= 4.0


def test_lwfa_window_full_of_plasma():
    """The measured workload: the same window with the ramp behind x = 0."""
    w = inputs.lwfa2d(ramp_x0=-8.0)
    q = w["particles"]
    assert len(q["x"]) == 2048 * 512 * 4 == 4_194_304
    assert np.all(q["w"] == 0.01 * 0.125 * 0.5 / 4)


def test_stress_counts_are_lognormal():
    """Per 16^3 block of the 256x128x128 grid: log-normal counts (sigma 1.5) summing to
    64M. Their max/mean of about 37 mirrors the paper's largest SP count of about 39
    times the initial one (Fig. 2)."""
    rng = np.random.default_rng(1513)
    c = inputs.lognormal_counts(16 * 8 * 8, 64 * 2 ** 20, 1.5, rng)
    assert c.sum() == 64 * 2 ** 20 and (c > 0).all()
    assert abs(np.log(c).std() - 1.5) < 0.1
    assert 30 < c.max() / c.mean() < 45
    # a small draw of the same generator: particles inside their blocks, momenta N(0, 0.05^2)
    w = inputs.stress3d(total=200_000)
    q = w["particles"]
    assert len(q["x"]) == 200_000
    L = [256 * 0.1, 128 * 0.1, 128 * 0.1]
    for a, k in enumerate(("x", "y", "z")):
        assert q[k].min() >= 0.0 and q[k].max() < L[a]
    assert abs(q["ux"].std() / 0.05 - 1.0) < 0.02
