"""Writes oracle_snapshots.json: summaries of the FP64 oracle's state after a few steps
of small seeded cases (2D/3D, periodic/moving window, Yee and sixth-order solver).

The paper prints no worked example whose numbers this method reproduces (its figures are
wall times and particle counts of full production runs), so no stored value here is the
paper's. These are regression snapshots of the oracle itself: they change only when the
oracle's arithmetic does, and such a change must name the passage that justifies it.
This script calls only `oracle` and the seeded input generators.

    python tests/golden/make_golden.py
"""
import json
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import oracle as orc  # noqa: E402
from paper_1511_03878_gb300 import inputs  # noqa: E402

OUT = os.path.join(HERE, "oracle_snapshots.json")


def cases():
    """(name, workload, steps) of the snapshot cases."""
    out = []
    for order, cfl in ((2, 0.95), (6, 0.76)):
        w = inputs.thermal2d(nx=32, ny=32, patch=(16, 16), cfl=cfl)
        out.append((f"thermal2d-32x32-order{order}", w, 10, order))
        w = inputs.lwfa2d(nx=128, ny=64, ppc=(2, 2), ramp_cells=16, w0=8.0, tau=6.0,
                          laser_back=10.0, patch=(16, 16), cfl=cfl)
        w = inputs.lwfa2d(nx=128, ny=64, ppc=(2, 2), ramp_cells=16, w0=8.0, tau=6.0,
                          laser_back=10.0, patch=(16, 16), cfl=cfl,
                          ramp_x0=w["params"]["xc"] - 6.0)
        out.append((f"lwfa2d-128x64-window-order{order}", w, 12, order))
        w = inputs.stress3d(n=(16, 8, 8), patch=(8, 8, 8), total=4000, cfl=cfl)
        out.append((f"stress3d-16x8x8-order{order}", w, 5, order))
    w = inputs.lwfa3d(nx=32, ny=8, nz=8, ppc=(1, 1, 1), laser_back=4.0, w0=2.0, tau=2.0,
                      ramp_cells=4, patch=(16, 8, 8))
    w = inputs.lwfa3d(nx=32, ny=8, nz=8, ppc=(1, 1, 1), laser_back=4.0, w0=2.0, tau=2.0,
                      ramp_cells=4, patch=(16, 8, 8), ramp_x0=w["params"]["xc"] - 4.0)
    out.append(("lwfa3d-32x8x8-window-order2", w, 6, 2))
    return out


def snapshot(w, steps, order):
    p = w["params"]
    dims = p["dims"]
    c = orc.make_config(dims, p["n"][:dims], p["d"][:dims], p["dt"], window=p["window"],
                        q=p["q"], m=p["m"], n0=p["n0"], ramp_x0=p["ramp_x0"],
                        ramp_len=p["ramp_len"], inject_ppc=p["inject_ppc"], order=order)
    o = orc.OracleSim(c, 4 * len(w["particles"]["x"]) + 20000)
    o.set_particles(w["particles"])
    o.set_fields(w["E"], w["B"])
    o.set_rho_bg(None)
    o.step(steps)
    f = o.get_fields()
    q = o.get_particles()
    snap = {"steps": steps, "shifts": int(o.shifts), "particles": int(len(q["id"])),
            "energy": [float(v) for v in o.energy()]}
    for k in ("Ex", "Ey", "Ez", "Bx", "By", "Bz", "Jx", "Jy", "Jz"):
        a = f[k]
        snap[k] = [float(np.abs(a).sum()), float((a * a).sum())]
    for k in ("x", "y", "z", "ux", "uy", "uz", "w"):
        if k in q:
            snap["p_" + k] = float(np.sum(q[k] * (1.0 + 1e-3 * q["id"])))
    snap["id_sum"] = int(np.sum(q["id"].astype(np.int64)))
    return snap


def main():
    orc.build()
    data = {name: snapshot(w, steps, order) for name, w, steps, order in cases()}
    with open(OUT, "w") as fh:
        json.dump(data, fh, indent=1, sort_keys=True)
    print(f"wrote {OUT}: {len(data)} cases")


if __name__ == "__main__":
    main()
