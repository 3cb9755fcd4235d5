"""GPU (CUDA, sm_103a) vs CPU FP64 oracle, element by element, through the C ABI.

Tolerances (normwise per array, max|a - b| / max|b|, particles matched by id):
  FP64, 1 step   : 1e-12     FP64, <= 20 steps : 1e-9
  FP32 (FP64 J)  : stated error, gated loosely (see each test).
"""
import math

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


def wrapdiff(a, b, L):
    return (a - b + 0.5 * L) % L - 0.5 * L


def make_oracle(w, cap=None):
    p = w["params"]
    c = orc.make_config(p["dims"], p["n"][:p["dims"]], p["d"][:p["dims"]], p["dt"],
                        window=p["window"], q=p["q"], m=p["m"], n0=p["n0"],
                        ramp_x0=p["ramp_x0"], ramp_len=p["ramp_len"],
                        inject_ppc=p["inject_ppc"])
    n = len(w["particles"]["x"])
    o = orc.OracleSim(c, cap or max(4 * n, 100000))
    o.set_particles(w["particles"])
    o.set_fields(w["E"], w["B"])
    o.set_rho_bg(None)
    return o


def compare(sim, o, params, tol, keys=FIELD_KEYS, check_particles=True):
    f = sim.fields()
    fo = o.get_fields()
    errs = {}
    for k in keys:
        errs[k] = normwise(f[k], fo[k])
    if check_particles:
        q = sim.particles()
        qo = o.get_particles()
        assert len(q["id"]) == len(qo["id"])
        assert np.array_equal(q["id"], qo["id"])
        Lx = params["n"][0] * params["d"][0]
        Ly = params["n"][1] * params["d"][1]
        dx = wrapdiff(q["x"], qo["x"], Lx) if not params["window"] else q["x"] - qo["x"]
        dy = wrapdiff(q["y"], qo["y"], Ly)
        errs["x"] = float(np.abs(dx).max() / max(np.abs(qo["x"]).max(), 1e-300))
        errs["y"] = float(np.abs(dy).max() / max(np.abs(qo["y"]).max(), 1e-300))
        for k in ("ux", "uy", "uz", "w"):
            errs[k] = normwise(q[k], qo[k])
    bad = {k: v for k, v in errs.items() if not (v <= tol)}
    assert not bad, (bad, errs)
    return errs


def small_lwfa(**kw):
    args = dict(nx=256, ny=128, dx=0.125, dy=0.5, ppc=(2, 2), n0=0.01, ramp_cells=16,
                a0=4.0, w0=15.0, tau=8.0, laser_back=12.0, patch=(32, 32))
    args.update(kw)
    w = inputs.lwfa2d(**args)
    # plasma already around the pulse: ramp from 8 units behind the laser centre
    if "ramp_x0" not in kw:
        w = inputs.lwfa2d(**args, ramp_x0=w["params"]["xc"] - 8.0)
    return w


# ------------------------------------------------------------------ FP64 parity

PREC64 = {"fp64": 0, "df64": 2}  # IEEE FP64 and double-word FP32 pairs: same tolerances


@pytest.mark.parametrize("prec", ["fp64", "df64"])
@pytest.mark.parametrize("steps,tol", [(1, 1e-12), (20, 1e-9)])
def test_thermal_fp64_full_size(binding, steps, tol, prec):
    """The thermal plasma at full size: 128x128, 16 ppc (262 144 particles)."""
    w = inputs.thermal2d(seed=1511)
    n = len(w["particles"]["x"])
    sim = binding.Sim(w["params"], precision=PREC64[prec], capacity=2 * n)
    sim.load(w)
    sim.step(steps)
    o = make_oracle(w)
    o.step(steps)
    compare(sim, o, w["params"], tol)
    assert sim.step_info() == (steps, 0)


@pytest.mark.parametrize("prec", ["fp64", "df64"])
@pytest.mark.parametrize("steps,tol", [(1, 1e-12), (20, 1e-9)])
def test_lwfa_small_fp64_window(binding, steps, tol, prec):
    """Moving window + injection + laser: shrunk LWFA (256x128, same dx, dy, dt)."""
    w = small_lwfa()
    n = len(w["particles"]["x"])
    sim = binding.Sim(w["params"], precision=PREC64[prec], capacity=8 * n + 100000)
    sim.load(w)
    sim.step(steps)
    o = make_oracle(w)
    o.step(steps)
    compare(sim, o, w["params"], tol)
    s, k = sim.step_info()
    assert s == steps and k == o.shifts == orc.shift_count(o.c, steps)


def test_patch_size_and_chunking_variants(binding):
    """Several tiles, ragged chunks and both work mappings give the same answer."""
    w = inputs.thermal2d(nx=96, ny=64, d=0.1, ppc_side=3, uth=0.1, seed=5, patch=(16, 32))
    n = len(w["particles"]["x"])
    o = make_oracle(w)
    o.step(3)
    for chunk, mapping in ((0, 0), (100, 0), (977, 0), (0, 1)):
        sim = binding.Sim(w["params"], precision=binding.PIC_FP64, capacity=2 * n,
                          chunk=chunk, mapping=mapping)
        sim.load(w)
        sim.step(3)
        compare(sim, o, w["params"], 1e-11)
        sim.close()


@pytest.mark.parametrize("prec", ["fp64", "df64"])
def test_gauss_law_on_gpu(binding, prec):
    """Esirkepov + Yee keep div E - rho at round-off on the GPU too (100 steps)."""
    w = inputs.thermal2d(nx=64, ny=64, d=0.1, uth=0.1, seed=8, patch=(16, 16))
    n = len(w["particles"]["x"])
    sim = binding.Sim(w["params"], precision=PREC64[prec], capacity=2 * n)
    sim.load(w)
    g0 = sim.gauss()
    assert np.abs(g0).max() < 1e-12
    sim.step(100)
    g = sim.gauss()
    assert np.abs(g - g0).max() < 1e-11
    assert np.abs(sim.fields()["Ex"]).max() > 1e-4


def test_energy_diag_matches_oracle(binding):
    w = inputs.thermal2d(nx=64, ny=64, d=0.1, seed=9, patch=(16, 16))
    n = len(w["particles"]["x"])
    sim = binding.Sim(w["params"], precision=binding.PIC_FP64, capacity=2 * n)
    sim.load(w)
    sim.step(10)
    o = make_oracle(w)
    o.step(10)
    e, eo = sim.energy(), o.energy()
    assert np.allclose(e, eo, rtol=1e-10, atol=1e-14)


# ------------------------------------------------------------------ edge cases

def _as_stored(v, prec):
    """A FP64 value as a precision stores it and reads back: FP32 rounds to float32,
    double-word keeps a float32 pair (hi, lo = v - hi rounded)."""
    if prec == 0:
        return v
    hi = v.astype(np.float32)
    if prec == 1:
        return hi.astype(np.float64)
    lo = (v - hi.astype(np.float64)).astype(np.float32)
    return hi.astype(np.float64) + lo.astype(np.float64)


def _position_as_stored(v, d, n, prec):
    """Read-back of a loaded position: c = v / d in cell units, kept below n (a value
    just under the domain's end can round to n); FP64 stores c, the cell precisions the
    cell floor(c) and the offset, kept below 1 when its rounding reaches 1."""
    c = v / d
    c = np.where(c >= n, np.nextafter(float(n), 0.0), c)
    if prec == 0:
        return c * d
    i = np.floor(c)
    f = c - i
    hi = f.astype(np.float32)
    below = float(np.nextafter(np.float32(1.0), np.float32(0.0)))
    return (i + np.where(hi >= 1.0, below, _as_stored(f, prec))) * d


# every precision in 2D; FP64 and FP32 in 3D (the double-word precision is 2D only)
@pytest.mark.parametrize("prec,dims", [(0, 2), (1, 2), (2, 2), (0, 3), (1, 3)])
@pytest.mark.parametrize("capfactor", [1, 4])
def test_load_places_and_converts_every_particle(binding, prec, dims, capfactor):
    """The device converts the caller's FP64 arrays during the load, in chunks of the
    repack scratch; FP32 at a capacity of n takes two. It also pads the fields. Read
    back right after the load, every particle is present once. Its position, momenta
    and weight match the precision's storage rule, including the conversion's edge
    cases: the domain's origin, a cell face, a position whose offset rounds to 1 in
    float32, and one just under the domain's end whose cell coordinate rounds to n.
    The fields come back as given, and the on-axis diagnostic is their Ex row."""
    if dims == 2:
        w = inputs.thermal2d(nx=64, ny=48, d=0.65, seed=3, patch=(16, 16))
    else:
        w = inputs.stress3d(n=(32, 16, 16), d=0.65, patch=(8, 8, 8), total=30000, seed=5)
    par = w["params"]
    q0 = {k: np.array(v, copy=True) for k, v in w["particles"].items()}
    keys = ("x", "y", "z")[:dims]
    for a, k in enumerate(keys):
        n_a, d_a = par["n"][a], par["d"][a]
        q0[k][0] = 0.0
        q0[k][1] = 3 * d_a
        q0[k][2] = np.nextafter(n_a * d_a, 0.0)
        q0[k][3] = (7 + (1 - 2.0 ** -30)) * d_a
    if dims == 2:  # 48 cells of 0.65: the position just under the end rounds to 48 cells
        assert q0["y"][2] / 0.65 >= 48
    rng = np.random.default_rng(11)
    E = [rng.normal(size=w["E"][0].shape) for _ in range(3)]
    B = [rng.normal(size=w["B"][0].shape) for _ in range(3)]
    n = len(q0["x"])
    sim = binding.Sim(par, precision=prec, capacity=capfactor * n)
    try:
        sim.load(dict(w, particles=q0, E=E, B=B))
        q = sim.particles()
        f = sim.fields()
        axis = sim.ex_axis()
    finally:
        sim.close()
    # the axis diagnostic reads the row (ny/2, nz/2) of Ex alone
    row = f["Ex"][par["n"][1] // 2] if dims == 2 else f["Ex"][par["n"][2] // 2, par["n"][1] // 2]
    assert np.array_equal(axis, row)
    assert np.array_equal(q["id"], np.sort(q0["id"]))
    order = np.argsort(q0["id"])
    for a, k in enumerate(keys):
        want = _position_as_stored(q0[k][order], par["d"][a], par["n"][a], prec)
        assert np.array_equal(q[k], want), k
    for k in ("ux", "uy", "uz", "w"):
        assert np.array_equal(q[k], _as_stored(q0[k][order], prec)), k
    for a, c in enumerate("xyz"):
        assert np.array_equal(f["E" + c], _as_stored(E[a], prec))
        assert np.array_equal(f["B" + c], _as_stored(B[a], prec))
        assert np.array_equal(f["Bn" + c], _as_stored(B[a], prec))
        assert not f["J" + c].any()


def test_empty_and_single_particle(binding):
    w = inputs.thermal2d(nx=32, ny=32, d=0.1, seed=1, patch=(16, 16))
    empty = {k: v[:0] for k, v in w["particles"].items()}
    sim = binding.Sim(w["params"], precision=binding.PIC_FP64, capacity=1000)
    sim.load(dict(w, particles=empty))
    sim.step(5)
    assert sim.num_particles() == 0
    assert np.abs(sim.fields()["Jx"]).max() == 0.0
    sim.close()
    # one fast particle crossing patch corners diagonally, periodic wrap
    one = dict(x=np.array([1.599]), y=np.array([1.599]), z=np.zeros(1),
               ux=np.array([3.0]), uy=np.array([3.0]), uz=np.array([0.5]),
               w=np.array([0.01]), id=np.array([7], np.int32))
    w1 = dict(w, particles=one)
    sim = binding.Sim(w["params"], precision=binding.PIC_FP64, capacity=1000)
    sim.load(w1)
    o = make_oracle(w1)
    for _ in range(6):
        sim.step(5)
        o.step(5)
        compare(sim, o, w["params"], 1e-10)


def test_one_heavy_patch(binding):
    """Most particles in one patch: chunked queue vs static mapping, same result."""
    rng = np.random.default_rng(4)
    N = 40000
    x = np.concatenate([rng.uniform(0.0, 1.6, N - 2000), rng.uniform(0, 6.4, 2000)])
    y = np.concatenate([rng.uniform(0.0, 1.6, N - 2000), rng.uniform(0, 6.4, 2000)])
    p = dict(x=x, y=y, z=np.zeros(N), ux=rng.normal(0, 0.1, N), uy=rng.normal(0, 0.1, N),
             uz=rng.normal(0, 0.1, N), w=np.full(N, 1e-3), id=np.arange(N, dtype=np.int32))
    w = inputs.thermal2d(nx=64, ny=64, d=0.1, seed=2, patch=(16, 16))
    w = dict(w, particles=p)
    o = make_oracle(w)
    o.step(4)
    for mapping in (0, 1):
        sim = binding.Sim(w["params"], precision=binding.PIC_FP64, capacity=3 * N,
                          chunk=512, mapping=mapping)
        sim.load(w)
        sim.step(4)
        compare(sim, o, w["params"], 1e-10)
        counts = sim.patch_counts()
        assert counts.sum() == N and counts.max() > 30000
        sim.close()


def test_repack_under_uneven_load(binding):
    """A dense blob next to empty patches with tight capacity: the device re-splits the
    per-patch capacities (repack) instead of overflowing, and results stay exact."""
    rng = np.random.default_rng(6)
    N = 30000
    x = rng.uniform(1.6, 3.2, N)
    y = rng.uniform(1.6, 3.2, N)
    p = dict(x=x, y=y, z=np.zeros(N), ux=rng.normal(0, 0.3, N), uy=rng.normal(0, 0.3, N),
             uz=rng.normal(0, 0.1, N), w=np.full(N, 1e-3), id=np.arange(N, dtype=np.int32))
    w = inputs.thermal2d(nx=64, ny=64, d=0.1, seed=2, patch=(16, 16))
    w = dict(w, particles=p)
    o = make_oracle(w)
    o.step(15)
    for prec in ("f64", "f32"):
        sim = binding.Sim(w["params"], precision=binding.PIC_FP64 if prec == "f64" else binding.PIC_FP32,
                          capacity=int(1.15 * N), chunk=700)
        sim.load(w)
        sim.step(15)
        sim.sync()
        assert sim.repacks() >= 1
        if prec == "f64":
            compare(sim, o, w["params"], 1e-9)
        else:
            q, qo = sim.particles(), o.get_particles()
            assert np.array_equal(q["id"], qo["id"])
            assert normwise(q["ux"], qo["ux"]) < 1e-4
        sim.close()


def test_capacity_overflow_is_reported(binding):
    """More particles than the arena holds (window injection into a half-empty box):
    the device latches PIC_ERR_CAPACITY; nothing faults."""
    w = small_lwfa()
    n = len(w["particles"]["x"])
    sim = binding.Sim(w["params"], precision=binding.PIC_FP64, capacity=n + 300)
    sim.load(w)
    sim.step(6)  # each shift injects 128 x 4 = 512 particles, few leave on the left
    with pytest.raises(binding.PicError) as e:
        sim.sync()
    assert e.value.code == binding.PIC_ERR_CAPACITY


def test_invalid_particles_rejected(binding):
    w = inputs.thermal2d(nx=32, ny=32, d=0.1, seed=1, patch=(16, 16))
    p = dict(w["particles"])
    p["x"] = p["x"].copy()
    p["x"][3] = 99.0
    sim = binding.Sim(w["params"], precision=binding.PIC_FP64, capacity=2 * len(p["x"]))
    with pytest.raises(binding.PicError) as e:
        binding.pic_load_particles(sim.h, p)
    assert e.value.code == binding.PIC_ERR_INVALID
    p["x"][3] = 0.5
    p["ux"] = p["ux"].copy()
    p["ux"][5] = np.nan
    with pytest.raises(binding.PicError) as e:
        binding.pic_load_particles(sim.h, p)
    assert e.value.code == binding.PIC_ERR_NUMERIC
    # a rejected load leaves the sim usable: the valid workload loads and steps as the
    # oracle does
    sim.load(w)
    sim.step(1)
    o = make_oracle(w)
    o.step(1)
    compare(sim, o, w["params"], 1e-12)
    sim.close()


@pytest.mark.parametrize("prec,capfactor", [(0, 2), (1, 1)])
def test_load_from_pinned_host_memory(binding, prec, capfactor):
    """Page-locked host arrays take the asynchronous copy path of the load (the
    first chunk overlapping the host's binning); the loaded state equals the one from
    pageable arrays bit for bit. FP32 at a capacity of n covers the later chunks. (After
    steps, the FP64 atomics of the current flush make runs differ in the last bits.)"""
    import torch

    w = inputs.thermal2d(nx=64, ny=64, d=0.1, seed=9, patch=(16, 16))
    keep = []

    def pinned(a):
        t = torch.empty(a.shape, dtype=torch.from_numpy(np.ascontiguousarray(a)).dtype,
                        pin_memory=True)
        keep.append(t)
        out = t.numpy()
        out[...] = a
        return out

    wp = dict(w, particles={k: pinned(v) for k, v in w["particles"].items()},
              E=[pinned(a) for a in w["E"]], B=[pinned(a) for a in w["B"]])
    n = len(w["particles"]["x"])
    got = []
    for work in (w, wp):
        sim = binding.Sim(w["params"], precision=prec, capacity=capfactor * n)
        sim.load(work)
        got.append((sim.particles(), sim.fields()))
        sim.close()
    (qa, fa), (qb, fb) = got
    for k in qa:
        assert np.array_equal(qa[k], qb[k]), k
    for k in fa:
        assert np.array_equal(fa[k], fb[k]), k


# ------------------------------------------------------------------ FP32 path

def test_thermal_fp32_error_stated(binding):
    """FP32 particles/fields, FP64 J: error against the FP64 oracle after 20 steps."""
    w = inputs.thermal2d(nx=64, ny=64, d=0.1, seed=12, patch=(16, 16))
    n = len(w["particles"]["x"])
    sim = binding.Sim(w["params"], precision=binding.PIC_FP32, capacity=2 * n)
    sim.load(w)
    sim.step(20)
    o = make_oracle(w)
    o.step(20)
    q, qo = sim.particles(), o.get_particles()
    assert np.array_equal(q["id"], qo["id"])
    ux_err = normwise(q["ux"], qo["ux"])
    x_err = np.abs(wrapdiff(q["x"], qo["x"], 6.4)).max() / 0.1  # in cells
    f, fo = sim.fields(), o.get_fields()
    ex_err = normwise(f["Ex"], fo["Ex"])
    print(f"FP32 thermal 20 steps: ux {ux_err:.2e}, x {x_err:.2e} cells, Ex {ex_err:.2e}")
    assert ux_err < 1e-4 and x_err < 1e-4 and ex_err < 1e-2
    e, eo = sim.energy(), o.energy()
    assert abs(e.sum() - eo.sum()) / eo.sum() < 1e-3


def test_lwfa_fp32_window(binding):
    w = small_lwfa()
    n = len(w["particles"]["x"])
    sim = binding.Sim(w["params"], precision=binding.PIC_FP32, capacity=8 * n + 100000)
    sim.load(w)
    sim.step(20)
    o = make_oracle(w)
    o.step(20)
    assert sim.num_particles() == o.num_particles()
    f, fo = sim.fields(), o.get_fields()
    ey_err = normwise(f["Ey"], fo["Ey"])
    e, eo = sim.energy(), o.energy()
    print(f"FP32 LWFA 20 steps: Ey {ey_err:.2e}, energy {abs(e.sum() / eo.sum() - 1):.2e}")
    assert ey_err < 1e-4
    assert abs(e.sum() - eo.sum()) / eo.sum() < 1e-3


# ------------------------------------------------------------------ 3D3V

def stress3d_small(seed=13, total=40000, patch=(8, 8, 8)):
    """32^3 slice with the statistics of the 3D stress case: log-normal counts over
    16^3 blocks (sigma = 1.5), uniform positions, u_th = 0.05; 8^3 patches."""
    w = inputs.stress3d(n=(32, 32, 32), d=0.1, patch=(16, 16, 16), total=total, sigma=1.5,
                        uth=0.05, seed=seed)
    w["params"] = dict(w["params"], patch=patch)
    return w


def compare3d(sim, o, params, tol):
    errs = compare(sim, o, params, tol)
    q, qo = sim.particles(), o.get_particles()
    Lz = params["n"][2] * params["d"][2]
    ez = float(np.abs(wrapdiff(q["z"], qo["z"], Lz)).max() / np.abs(qo["z"]).max())
    assert ez <= tol, ez
    return errs


@pytest.mark.parametrize("prec", ["fp64"])  # the double-word precision is 2D only
@pytest.mark.parametrize("steps,tol", [(1, 1e-12), (10, 1e-9)])
def test_stress3d_fp64(binding, steps, tol, prec):
    w = stress3d_small()
    n = len(w["particles"]["x"])
    sim = binding.Sim(w["params"], precision=PREC64[prec], capacity=2 * n)
    sim.load(w)
    sim.step(steps)
    o = make_oracle(w)
    o.step(steps)
    compare3d(sim, o, w["params"], tol)


def test_stress3d_static_mapping_and_chunks(binding):
    w = stress3d_small(seed=14)
    n = len(w["particles"]["x"])
    o = make_oracle(w)
    o.step(3)
    for chunk, mapping in ((300, 0), (0, 1)):
        sim = binding.Sim(w["params"], precision=binding.PIC_FP64, capacity=2 * n, chunk=chunk,
                          mapping=mapping)
        sim.load(w)
        sim.step(3)
        compare3d(sim, o, w["params"], 1e-11)
        sim.close()


def test_gauss_law_3d_gpu(binding):
    w = stress3d_small(seed=15, total=20000)
    n = len(w["particles"]["x"])
    sim = binding.Sim(w["params"], precision=binding.PIC_FP64, capacity=2 * n)
    sim.load(w)
    g0 = sim.gauss()
    sim.step(30)
    assert np.abs(sim.gauss() - g0).max() < 1e-10


def test_stress3d_fp32_error_stated(binding):
    w = stress3d_small(seed=16)
    n = len(w["particles"]["x"])
    sim = binding.Sim(w["params"], precision=binding.PIC_FP32, capacity=2 * n)
    sim.load(w)
    sim.step(10)
    o = make_oracle(w)
    o.step(10)
    q, qo = sim.particles(), o.get_particles()
    assert np.array_equal(q["id"], qo["id"])
    ux_err = normwise(q["ux"], qo["ux"])
    f, fo = sim.fields(), o.get_fields()
    jx_err = normwise(f["Jx"], fo["Jx"])
    e, eo = sim.energy(), o.energy()
    print(f"FP32 3D 10 steps: ux {ux_err:.2e}, Jx {jx_err:.2e}, "
          f"energy {abs(e.sum() / eo.sum() - 1):.2e}")
    assert ux_err < 1e-4 and jx_err < 1e-3
    assert abs(e.sum() - eo.sum()) / eo.sum() < 1e-3


@pytest.mark.parametrize("mapping,chunk", [(1, 0), (0, 16384)])
def test_more_leavers_than_the_shared_list(binding, mapping, chunk):
    """4x4 patches of 4096 particles (256 per cell), fast thermal particles (u_th = 1):
    about 530 particles leave each patch per step, and with one work item per patch
    (static mapping, or a chunk above the patch count) more than the 512 an item lists
    in shared memory; the rest take the hand-off inside the particle loop. FP64 against
    the oracle after 3 steps."""
    w = inputs.thermal2d(nx=32, ny=32, ppc_side=16, uth=1.0, seed=9, patch=(4, 4))
    n = len(w["particles"]["x"])
    o = make_oracle(w)
    o.step(3)
    sim = binding.Sim(w["params"], precision=binding.PIC_FP64, capacity=3 * n, chunk=chunk,
                      mapping=mapping)
    sim.load(w)
    sim.step(3)
    compare(sim, o, w["params"], 1e-9)
    assert sim.num_particles() == n
    sim.close()
