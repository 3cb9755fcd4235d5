"""The oracle's threaded step (orc_step_mt) against its plain step (orc_step): the
results must be identical bit for bit (fields, current, particles, counters), on 2D
and 3D, periodic and moving-window grids, both solver orders, and thread counts whose
bands of J rows are narrower than the 5-node deposit stencil. The threaded form is
what the long-run precision sweep and the all-core CPU baseline use."""
import numpy as np
import pytest

import oracle as orc
from paper_1511_03878_gb300 import inputs


def _oracle(w, order=2):
    p = w["params"]
    c = orc.make_config(p["dims"], p["n"][:p["dims"]], p["d"][:p["dims"]], p["dt"],
                        window=p["window"], q=p["q"], m=p["m"], n0=p["n0"],
                        ramp_x0=p["ramp_x0"], ramp_len=p["ramp_len"],
                        inject_ppc=p["inject_ppc"], order=order)
    o = orc.OracleSim(c, 4 * len(w["particles"]["x"]) + 20000)
    o.set_particles(w["particles"])
    o.set_fields(w["E"], w["B"])
    o.set_rho_bg(None)
    return o


def _same(a, b):
    fa, fb = a.get_fields(), b.get_fields()
    for k in fa:
        assert np.array_equal(fa[k], fb[k]), k
    pa, pb = a.get_particles(sort_by_id=False), b.get_particles(sort_by_id=False)
    for k in pa:
        assert np.array_equal(pa[k], pb[k]), k
    assert a.steps == b.steps and a.shifts == b.shifts
    assert np.array_equal(a.energy(), b.energy())
    assert np.array_equal(a.gauss(), b.gauss())


def _cases():
    lw = inputs.lwfa2d(nx=128, ny=32, dx=0.125, dy=0.5, ppc=(2, 2), n0=0.01, ramp_cells=16,
                       a0=4.0, w0=6.0, tau=5.0, laser_back=10.0, ramp_x0=2.0, patch=(16, 16))
    th = inputs.thermal2d(nx=32, ny=16, d=0.1, ppc_side=3, uth=0.2, seed=7, patch=(16, 16))
    s3 = inputs.stress3d(n=(16, 8, 12), patch=(8, 4, 4), total=3000, seed=9)
    l3 = inputs.lwfa3d(nx=32, ny=8, nz=8, patch=(16, 8, 8))
    return [("lwfa2d", lw, 2, 12), ("thermal2d", th, 2, 10), ("thermal2d-o6", th, 6, 6),
            ("stress3d", s3, 2, 5), ("lwfa3d", l3, 2, 9), ("lwfa2d-o6", lw, 6, 8)]


@pytest.mark.parametrize("threads", [3, 8])
@pytest.mark.parametrize("case", range(6))
def test_threaded_oracle_is_bit_identical(case, threads):
    name, w, order, steps = _cases()[case]
    a = _oracle(w, order)
    b = _oracle(w, order)
    a.step(steps)
    b.step(steps, threads=threads)
    _same(a, b)
    if w["params"]["window"]:
        assert a.shifts > 0, name
