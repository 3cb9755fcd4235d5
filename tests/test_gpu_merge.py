"""Load limiting by particle merging on the GPU, against the oracle's merge (same rule,
same free choices) and against the conservation laws it must keep."""
import numpy as np
import pytest

import oracle as orc
from paper_1511_03878_gb300 import inputs

pytestmark = pytest.mark.gpu

FIELD_KEYS = ("Ex", "Ey", "Ez", "Bx", "By", "Bz", "Jx", "Jy", "Jz")


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


def hot_workload(seed=21, dims=2):
    """Periodic box, 16^dims-cell patches; three cells of the first patch hold 300
    particles each with momenta clustered around u_x = 0.3, the rest 3 per cell with
    thermal momenta; zero initial fields."""
    rng = np.random.default_rng(seed)
    d = 0.1
    n = (32, 32, 32)[:dims]
    P = (16, 16, 16)[:dims] if dims == 2 else (8, 8, 8)
    xs = [[] for _ in range(3)]
    us = []
    for cc in ((1, 1, 1), (2, 1, 1), (5, 6, 2))[:3]:
        m = 300
        for a in range(dims):
            xs[a].append((cc[a] + rng.random(m)) * d)
        us.append(rng.normal([[0.3], [0.0], [0.0]], 0.06, (3, m)))
    grid = np.stack(np.meshgrid(*[np.arange(v) for v in n], indexing="ij"), axis=-1).reshape(-1, dims)
    for c in grid:
        for a in range(dims):
            xs[a].append((c[a] + rng.random(3)) * d)
        us.append(rng.normal(0.0, 0.05, (3, 3)))
    pos = [np.concatenate(x) for x in xs[:dims]]
    u = np.concatenate(us, axis=1)
    N = len(pos[0])
    parts = dict(x=pos[0], y=pos[1], z=pos[2] if dims == 3 else np.zeros(N), ux=u[0].copy(),
                 uy=u[1].copy(), uz=u[2].copy(), w=rng.uniform(0.5, 1.5, N) * 0.01,
                 id=rng.permutation(N).astype(np.int32))
    dt = inputs.cfl_dt((d,) * dims)
    params = dict(dims=dims, n=n, d=(d,) * dims, dt=dt, window=False, q=-1.0, m=1.0, n0=0.0,
                  ramp_x0=0.0, ramp_len=1.0, inject_ppc=(1, 1, 1), patch=P)
    shp = tuple(reversed(n))
    return dict(params=params, particles=parts, E=[np.zeros(shp)] * 3, B=[np.zeros(shp)] * 3)


def oracle_run(w, steps, above, dp):
    p = w["params"]
    c = orc.make_config(p["dims"], p["n"], p["d"], p["dt"], q=p["q"], m=p["m"])
    o = orc.OracleSim(c, len(w["particles"]["x"]))
    o.set_particles(w["particles"])
    o.set_fields(w["E"], w["B"])
    o.set_rho_bg(None)
    removed = 0
    for _ in range(steps):
        o.step(1)
        removed += o.merge(p["patch"], above, dp)
    return o, removed


@pytest.mark.parametrize("dims", [2, 3])
@pytest.mark.parametrize("steps,tol", [(1, 1e-12), (4, 1e-9)])
def test_merge_matches_oracle(binding, dims, steps, tol):
    w = hot_workload(dims=dims)
    above, dp = (1000 if dims == 2 else 2000), 0.05  # only the hot patch is above
    n0 = len(w["particles"]["x"])
    sim = binding.Sim(w["params"], precision=binding.PIC_FP64, capacity=2 * n0,
                      merge_above=above, merge_dp=dp)
    sim.load(w)
    sim.step(steps)
    o, removed = oracle_run(w, steps, above, dp)
    assert removed > 0
    assert sim.merged() == removed
    q, qo = sim.particles(), o.get_particles()
    assert np.array_equal(q["id"], qo["id"])
    for k in ("x", "y", "ux", "uy", "uz", "w"):
        assert normwise(q[k], qo[k]) < tol, k
    f, fo = sim.fields(), o.get_fields()
    for k in FIELD_KEYS:
        assert normwise(f[k], fo[k]) < tol, k
    sim.close()


@pytest.mark.parametrize("prec", ["fp64", "df64", "fp32"])
def test_merge_conserves_on_gpu(binding, prec):
    """With zero fields the first push leaves momenta unchanged, so the step's merge is
    the only change of total weight, momentum and energy, which it must keep."""
    w = hot_workload(seed=22)
    P = {"fp64": binding.PIC_FP64, "df64": binding.PIC_DF64, "fp32": binding.PIC_FP32}[prec]
    n0 = len(w["particles"]["x"])
    sim = binding.Sim(w["params"], precision=P, capacity=2 * n0, merge_above=400, merge_dp=0.05)
    sim.load(w)
    p0 = sim.particles()
    sim.step(1)
    p1 = sim.particles()
    assert sim.merged() > 0 and len(p1["id"]) == n0 - sim.merged()

    def tot(p):
        u = np.vstack([p["ux"], p["uy"], p["uz"]])
        return p["w"].sum(), (p["w"] * u).sum(axis=1), (p["w"] * np.sqrt(1 + (u ** 2).sum(0))).sum()

    (W0, P0, E0), (W1, P1, E1) = tot(p0), tot(p1)
    tol = 1e-12 if prec != "fp32" else 1e-6
    assert abs(W1 - W0) <= tol * W0
    assert np.abs(P1 - P0).max() <= tol * np.abs(p0["w"] * p0["ux"]).sum()
    assert abs(E1 - E0) <= tol * E0
    sim.close()


def test_merge_off_and_cold_patches_untouched(binding):
    w = hot_workload(seed=23)
    n0 = len(w["particles"]["x"])
    sim = binding.Sim(w["params"], precision=binding.PIC_FP64, capacity=2 * n0,
                      merge_above=100000, merge_dp=0.05)
    sim.load(w)
    sim.step(2)
    assert sim.merged() == 0 and sim.num_particles() == n0
    sim.close()
