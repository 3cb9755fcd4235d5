"""The allocation-free Gauss-residual entry point (pic_gauss_residual_2d_static).

It serves callers that cannot allocate device memory (code inside another
framework's memory pool or under a fixed device budget, where cudaMalloc would fail
or synchronise the device). It keeps its charge-density scratch in a static device
array instead. Each case compares it with the FP64 CPU oracle's Gauss residual
(orc_gauss) on the same particles and fields, and with the library's own
pic_diag(GAUSS) where a sim holds that state. This file is collected last, so that a
run that stops at the first failure has already run every other test.
"""
import numpy as np
import pytest

import oracle as orc

pytestmark = pytest.mark.gpu

TOL = 1e-12  # normwise, max|a - b| / max|b| (FP64: atomics reorder the charge sums)


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1511_03878_gb300 import binding, build, inputs

    build.build()
    return torch, binding, inputs


def _normwise(a, b):
    return float(np.abs(a - b).max() / np.abs(b).max())


def _oracle_gauss(p, parts, Ex, Ey, rho_bg):
    """orc_gauss on a given state: div E (two-point) - rho_e - rho_bg."""
    nx, ny = p["n"][0], p["n"][1]
    c = orc.make_config(2, (nx, ny), p["d"][:2], p["dt"], window=p["window"], q=p["q"],
                        m=p["m"])
    o = orc.OracleSim(c, max(len(parts["x"]), 1))
    o.set_particles(parts)
    z = np.zeros((ny, nx))
    o.set_fields([Ex, Ey, z], [z, z, z])
    o.set_rho_bg(rho_bg)
    return o.gauss()


def _call(env, p, parts, Ex, Ey, rho_bg, out):
    torch, binding, _ = env
    dev = lambda a: torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")
    x, y, wt = dev(parts["x"]), dev(parts["y"]), dev(parts["w"])
    ex, ey = dev(Ex), dev(Ey)
    rb = dev(rho_bg) if rho_bg is not None else None
    out.fill_(float("nan"))
    stream = torch.cuda.current_stream()
    rc = binding.pic_gauss_residual_2d_static(
        len(parts["x"]), x.data_ptr(), y.data_ptr(), wt.data_ptr(), p["q"], ex.data_ptr(),
        ey.data_ptr(), rb.data_ptr() if rb is not None else 0, out.data_ptr(), p["n"][0],
        p["n"][1], p["d"][0], p["d"][1], 1 if p["window"] else 0, stream.cuda_stream)
    assert rc == binding.PIC_OK
    torch.cuda.synchronize()
    return out.cpu().numpy().copy()


def test_static_gauss_residual_matches_oracle_and_diag(env):
    torch, binding, inputs = env
    nx = ny = 64
    w = inputs.thermal2d(nx=nx, ny=ny, d=0.1, uth=0.1, seed=21, patch=(16, 16))
    p = w["params"]
    n = len(w["particles"]["x"])
    sim = binding.Sim(p, precision=binding.PIC_FP64, capacity=2 * n)
    # no background: the residual is div E - rho_e, an O(1) field worth comparing
    sim.load(w, rho_bg=np.zeros((ny, nx)))
    sim.step(7)
    diag = sim.gauss()          # the existing entry point (pic_diag, PIC_DIAG_GAUSS)
    q = sim.particles()
    f = sim.fields()
    ref = _oracle_gauss(p, q, f["Ex"], f["Ey"], np.zeros((ny, nx)))
    assert np.abs(ref).max() > 0.1
    out = torch.empty((ny, nx), dtype=torch.float64, device="cuda")
    for call in range(2):  # two calls in a row: the shared scratch is cleared each time
        got = _call(env, p, q, f["Ex"], f["Ey"], None, out)
        assert _normwise(got, ref) < TOL, (call, _normwise(got, ref))
        assert _normwise(got, diag) < TOL, (call, _normwise(got, diag))
    # sizes beyond the static scratch are rejected before any launch
    dummy = torch.zeros(8, dtype=torch.float64, device="cuda")
    rc = binding.pic_gauss_residual_2d_static(
        n, dummy.data_ptr(), dummy.data_ptr(), dummy.data_ptr(), p["q"], dummy.data_ptr(),
        dummy.data_ptr(), 0, out.data_ptr(), 2048, 1024, p["d"][0], p["d"][1], 0,
        torch.cuda.current_stream().cuda_stream)
    assert rc == binding.PIC_ERR_NOMEM
    sim.close()


def test_static_gauss_residual_window_with_background(env):
    """Moving window (x taps outside [0, nx) dropped, Ex zero below i = 0) and an
    explicit background charge, on a shrunk LWFA window after several shifts."""
    torch, binding, inputs = env
    args = dict(nx=256, ny=128, dx=0.125, dy=0.5, ppc=(2, 2), n0=0.01, ramp_cells=16,
                a0=4.0, w0=15.0, tau=8.0, laser_back=12.0, patch=(32, 32))
    w0 = inputs.lwfa2d(**args)
    w = inputs.lwfa2d(**args, ramp_x0=w0["params"]["xc"] - 8.0)
    p = w["params"]
    nx, ny = p["n"][0], p["n"][1]
    pp = w["particles"]
    c = orc.make_config(2, (nx, ny), p["d"][:2], p["dt"], window=True)
    rho_bg = -orc.rho(c, pp["x"], pp["y"], None, pp["w"], p["q"])
    n = len(pp["x"])
    sim = binding.Sim(p, precision=binding.PIC_FP64, capacity=4 * n + 100000)
    sim.load(w, rho_bg=rho_bg)
    sim.step(9)
    assert sim.step_info()[1] >= 5  # the window has shifted
    diag = sim.gauss()
    q = sim.particles()
    f = sim.fields()
    ref = _oracle_gauss(p, q, f["Ex"], f["Ey"], rho_bg)
    out = torch.empty((ny, nx), dtype=torch.float64, device="cuda")
    for call in range(2):
        got = _call(env, p, q, f["Ex"], f["Ey"], rho_bg, out)
        assert _normwise(got, ref) < TOL, (call, _normwise(got, ref))
        assert _normwise(got, diag) < TOL, (call, _normwise(got, diag))
    sim.close()


def _edge_dx(nx):
    """A cell size for which the last double below nx dx, times the rounded reciprocal
    1/dx, rounds up to exactly nx (the position is inside the grid, its cell coordinate
    computed that way is not)."""
    for k in range(1, 200000):
        dx = 0.1 + k * 1.37e-7
        x = np.nextafter(nx * dx, 0.0)
        if x * (1.0 / dx) == nx and x < nx * dx:
            return dx, x
    raise AssertionError("no such dx found")


@pytest.mark.parametrize("window", [False, True])
def test_static_gauss_residual_particle_at_the_domain_end(env, window):
    torch, binding, _ = env
    nx, ny = 64, 32
    dx, xe = _edge_dx(nx)
    dy, ye = _edge_dx(ny)
    p = dict(n=(nx, ny, 1), d=(dx, dy, 1.0), dt=0.05, window=window, q=-1.0, m=1.0)
    rng = np.random.default_rng(4)
    m = 40
    x = rng.uniform(0, nx * dx, m)
    y = rng.uniform(0, ny * dy, m)
    x[:3] = [xe, xe, 0.5 * nx * dx]
    y[:3] = [0.5 * ny * dy, ye, ye]
    parts = dict(x=x, y=y, z=np.zeros(m), ux=np.zeros(m), uy=np.zeros(m), uz=np.zeros(m),
                 w=rng.uniform(0.5, 1.5, m), id=np.arange(m, dtype=np.int32))
    Ex = rng.standard_normal((ny, nx))
    Ey = rng.standard_normal((ny, nx))
    ref = _oracle_gauss(p, parts, Ex, Ey, np.zeros((ny, nx)))
    out = torch.empty((ny, nx), dtype=torch.float64, device="cuda")
    got = _call(env, p, parts, Ex, Ey, None, out)
    assert _normwise(got, ref) < TOL, _normwise(got, ref)
    # the edge particles' charge is there: without them the residual differs
    keep = np.arange(m) >= 3
    part3 = {k: v[keep] for k, v in parts.items()}
    ref3 = _oracle_gauss(p, part3, Ex, Ey, np.zeros((ny, nx)))
    assert _normwise(ref3, ref) > 1e-3
