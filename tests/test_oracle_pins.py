"""Pins of the FP64 CPU oracle against what the mathematics fixes (no GPU).

The paper prints no PIC equations and no worked example (Sec. 2.1 identifies only a
standard second-order field scheme), so each part of the oracle is pinned by a closed
form or an invariant of the published scheme it restates:
  * quadratic B-spline: partition of unity, first moment, variance 1/4, continuity;
  * Boris: |u| conservation, exact discrete rotation angle, gyration radius of the
    discrete orbit, rotation sense, E x B drift, relativistic uniform-E acceleration;
  * interpolation: exact reproduction of fields linear in position, per stagger;
  * Esirkepov: discrete continuity equation for one particle, zero current at rest,
    total current q w v / dV;
  * Yee: discrete dispersion relation of vacuum modes, dispersion-free 1D transport
    at dt = dx;
  * full step: Gauss's law preserved to round-off for 100 steps; a cold plasma mode
    oscillates at the plasma frequency;
  * energy diagnostic: closed-form field and kinetic energies;
  * charge density: its total and first two moments from the spline's moments;
  * moving window: shift count floor(n dt/dx), exact field translation, injection.
A plausible mistake anywhere (a dropped term, a sign, a stagger, a transposed
index) breaks at least one of these.
"""
import math

import numpy as np
import pytest

import oracle as orc
from paper_1511_03878_gb300 import inputs


# ------------------------------------------------------------------ shapes

def test_shape_moments_and_continuity():
    rng = np.random.default_rng(0)
    for xi in np.concatenate([rng.uniform(-50, 50, 500), [0.0, 0.5, -0.5, 3.5, 7.25]]):
        i, S = orc.shape2(xi)
        delta = xi - i
        assert -0.5 <= delta <= 0.5
        assert np.all(S >= 0)
        k = np.array([-1.0, 0.0, 1.0])
        assert abs(S.sum() - 1.0) < 1e-15
        assert abs((k * S).sum() - delta) < 1e-15            # first moment
        assert abs((((k - delta) ** 2) * S).sum() - 0.25) < 1e-15  # variance 1/4
    # continuity where the nearest node changes: weights per node agree
    for node in (-3, 0, 5):
        xl = node + 0.5 - 1e-13
        il, Sl = orc.shape2(xl)
        ir, Sr = orc.shape2(node + 0.5)
        wl = {il + a - 1: Sl[a] for a in range(3)}
        wr = {ir + a - 1: Sr[a] for a in range(3)}
        for n in set(wl) | set(wr):
            assert abs(wl.get(n, 0.0) - wr.get(n, 0.0)) < 1e-12


# ------------------------------------------------------------------ Boris

def test_boris_pure_b_rotation_exact():
    q, m, dt = -1.0, 1.0, 0.1
    B = np.array([0.3, -0.2, 1.7])
    E = np.zeros(3)
    u0 = np.array([0.8, -0.4, 0.25])
    u = u0.copy()
    gamma = math.sqrt(1 + u0 @ u0)
    Bm = np.linalg.norm(B)
    theta = 2 * math.atan(abs(q) * Bm * dt / (2 * m * gamma))
    bh = B / Bm
    upar = (u0 @ bh) * bh
    for n in range(1, 400):
        u = orc.boris(q, m, dt, E, B, u)
        assert abs(np.linalg.norm(u) - np.linalg.norm(u0)) < 1e-14 * n
    # after 399 steps the perpendicular part has turned by 399 theta around b
    n = 399
    uperp0 = u0 - upar
    uperp = u - (u @ bh) * bh
    cosang = (uperp0 @ uperp) / (np.linalg.norm(uperp0) * np.linalg.norm(uperp))
    # rotation sense: an electron gyrates right-handed about B (omega parallel to B)
    sin_signed = np.cross(uperp0, uperp) @ bh / (np.linalg.norm(uperp0) ** 2)
    ang = math.atan2(sin_signed, cosang)
    expect = math.remainder(n * theta, 2 * math.pi)
    assert abs(ang - expect) < 1e-11
    assert np.allclose(u @ bh, u0 @ bh, rtol=0, atol=1e-14)


def test_boris_single_step_angle_and_sense():
    q, m, dt = -1.0, 1.0, 0.05
    for Bz in (0.5, 2.0, 10.0):
        u0 = np.array([1.2, 0.0, 0.0])
        u1 = orc.boris(q, m, dt, np.zeros(3), np.array([0, 0, Bz]), u0)
        gamma = math.sqrt(1 + 1.2 ** 2)
        theta = 2 * math.atan(Bz * dt / (2 * gamma))
        # q < 0, B along +z: v = +x turns towards +y
        assert abs(math.atan2(u1[1], u1[0]) - theta) < 1e-15
        # q > 0 turns the other way
        u2 = orc.boris(1.0, m, dt, np.zeros(3), np.array([0, 0, Bz]), u0)
        assert abs(math.atan2(u2[1], u2[0]) + theta) < 1e-15


def _uniform_field_sim(E0, B0, n=(16, 16), d=(0.1, 0.1), dt=0.05):
    c = orc.make_config(2, n, d, dt)
    s = orc.OracleSim(c, 4)
    shp = (n[1], n[0])
    s.set_fields([np.full(shp, e) for e in E0], [np.full(shp, b) for b in B0])
    return c, s


def test_full_step_gyration_radius_period_and_drift():
    # one weightless electron in uniform Bz: interpolation + Boris + move
    Bz = 2.0
    dt = 0.05
    c, s = _uniform_field_sim((0, 0, 0), (0, 0, Bz), n=(64, 64), d=(0.1, 0.1), dt=dt)
    u0 = 0.3
    p = dict(x=np.array([3.2]), y=np.array([3.2]), z=np.zeros(1), ux=np.array([u0]),
             uy=np.zeros(1), uz=np.zeros(1), w=np.zeros(1), id=np.array([0], np.int32))
    s.set_particles(p)
    pts = []
    for _ in range(200):
        s.step(1)
        q = s.get_particles()
        pts.append((q["x"][0], q["y"][0]))
    pts = np.array(pts)
    gamma = math.sqrt(1 + u0 * u0)
    b = Bz * dt / (2 * gamma)
    # discrete orbit: regular polygon, side dt*v, exterior angle 2 atan b
    R_exact = (u0 / Bz) * math.sqrt(1 + b * b)
    # circle through the points: least squares
    A = np.c_[2 * pts[:, 0], 2 * pts[:, 1], np.ones(len(pts))]
    rhs = (pts ** 2).sum(1)
    cx, cy, k = np.linalg.lstsq(A, rhs, rcond=None)[0]
    R = math.sqrt(k + cx * cx + cy * cy)
    assert abs(R - R_exact) < 1e-11
    r = np.hypot(pts[:, 0] - cx, pts[:, 1] - cy)
    assert np.ptp(r) < 1e-11
    # period: angle advanced per step
    ang = np.unwrap(np.arctan2(pts[:, 1] - cy, pts[:, 0] - cx))
    step_ang = np.diff(ang)
    assert np.allclose(step_ang, 2 * math.atan(b), rtol=0, atol=1e-11)  # electron: +z sense
    # continuum limit O(dt^2): R_exact -> Larmor radius gamma v / (|q| B)
    assert abs(R_exact / (u0 / Bz) - 1) < (b * b)


def test_uniform_e_acceleration_follows_the_relativistic_trajectory():
    """A test particle (negligible weight) in a uniform Ex, with no B, starting at rest
    at t = -dt/2. Boris has no rotation here, so u^(N-1/2) = (q E / m) N dt exactly.
    The leapfrog positions follow the relativistic hyperbola
    x(t) = x0 + (sqrt(1 + a^2 (t + dt/2)^2) - sqrt(1 + a^2 dt^2/4)) / a, with a = q E / m,
    to second order in dt. The error falls by 4 when dt halves, out to u = 5. Dropping
    the 1/gamma of the move would put the particle several units off."""
    errs = []
    for dt in (0.05, 0.025):
        c = orc.make_config(2, (32, 32), (0.1, 0.1), dt)
        s = orc.OracleSim(c, 4)
        s.set_particles(dict(x=np.array([1.6]), y=np.array([1.6]), z=np.zeros(1),
                             ux=np.zeros(1), uy=np.zeros(1), uz=np.zeros(1),
                             w=np.array([1e-15]), id=np.zeros(1, np.int32)))
        zero = np.zeros((32, 32))
        s.set_fields([np.full((32, 32), 0.5), zero, zero], [zero, zero, zero])
        s.set_rho_bg(None)
        N = int(round(10.0 / dt))
        s.step(N)
        r = s.get_particles()
        a = -0.5  # q E / m for an electron
        assert abs(r["ux"][0] - a * N * dt) < 1e-12 * abs(a * N * dt)
        assert abs(r["uy"][0]) < 1e-15 and abs(r["uz"][0]) < 1e-15
        t = N * dt
        x = 1.6 + (math.sqrt(1 + (a * (t + dt / 2)) ** 2) - math.sqrt(1 + (a * dt / 2) ** 2)) / a
        errs.append(abs(((r["x"][0] - x + 1.6) % 3.2) - 1.6))  # periodic box of 3.2
    assert errs[0] < 1e-4
    assert 3.5 < errs[0] / errs[1] < 4.5


def test_e_cross_b_drift():
    Ey, Bz = 0.002, 1.0
    c, s = _uniform_field_sim((0, Ey, 0), (0, 0, Bz), n=(64, 64), d=(0.1, 0.1), dt=0.05)
    p = dict(x=np.array([3.2]), y=np.array([3.2]), z=np.zeros(1), ux=np.zeros(1),
             uy=np.zeros(1), uz=np.zeros(1), w=np.zeros(1), id=np.array([0], np.int32))
    s.set_particles(p)
    # integrate over an integer number of discrete gyro-periods
    theta = 2 * math.atan(Bz * 0.05 / 2)
    nper = 2 * math.pi / theta
    nsteps = int(round(20 * nper))
    x0 = 3.2
    xs = []
    for _ in range(nsteps):
        s.step(1)
        xs.append(s.get_particles()["x"][0])
    xs = np.unwrap(np.array(xs), period=6.4)
    vd = (xs[-1] - x0) / (nsteps * 0.05)
    # E x B / B^2 = (Ey Bz, 0, 0) / Bz^2 = +Ey/Bz along x; independent of charge
    assert abs(vd - Ey / Bz) < 2e-2 * Ey / Bz


# ------------------------------------------------------------------ interpolation

STAG = [(1, 0, 0), (0, 1, 0), (0, 0, 1), (0, 1, 1), (1, 0, 1), (1, 1, 0)]


@pytest.mark.parametrize("dims", [2, 3])
def test_interp_reproduces_linear_fields(dims):
    # window config: x has no wrap, so a field linear in x is exact away from edges
    n = (24, 8, 8 if dims == 3 else 1)
    d = (0.2, 0.3, 0.25)
    c = orc.make_config(dims, n[:dims], d[:dims], 0.05, window=True)
    shp = orc.field_shape(c)
    rng = np.random.default_rng(1)
    for comp in range(6):
        a, b = rng.uniform(-2, 2, 2)
        F = [np.zeros(shp) for _ in range(6)]
        i = np.arange(n[0])
        xpos = (i + 0.5 * STAG[comp][0]) * d[0]
        F[comp][...] = a + b * xpos  # broadcast over trailing x axis
        for _ in range(20):
            pos = [rng.uniform(5 * d[0], (n[0] - 5) * d[0]), rng.uniform(0, n[1] * d[1]),
                   rng.uniform(0, n[2] * d[2])]
            out = orc.interp(c, F, pos[:dims])
            assert abs(out[comp] - (a + b * pos[0])) < 1e-13
            others = [out[k] for k in range(6) if k != comp]
            assert max(abs(v) for v in others) == 0.0


def _stag_pos(n, d, comp, axis):
    """Positions of a component's stored values along one axis: index i sits at
    (i + s/2) d, s the component's stagger bit on that axis (Yee 1966)."""
    return (np.arange(n[axis]) + 0.5 * STAG[comp][axis]) * d[axis]


@pytest.mark.parametrize("window", [True, False])
@pytest.mark.parametrize("axis", [1, 2])
def test_interp_3d_reproduces_fields_linear_in_y_and_z(window, axis):
    # Quadratic B-splines reproduce linear functions exactly (first moment = delta), so
    # a 3D field linear along y or z comes back exactly at any position whose three taps
    # along that axis stay on the same side of the periodic seam -- but only if the
    # oracle uses each component's own y and z stagger. A wrong stagger bit shifts the
    # result by b d/2 (b the slope), far above the 1e-13 bound.
    n = (12, 16, 20)
    d = (0.2, 0.3, 0.25)
    c = orc.make_config(3, n, d, 0.05, window=window)
    shp = orc.field_shape(c)  # (nz, ny, nx)
    rng = np.random.default_rng(11 + axis + 2 * window)
    for comp in range(6):
        a, b = rng.uniform(-2, 2, 2)
        F = [np.zeros(shp) for _ in range(6)]
        coord = _stag_pos(n, d, comp, axis)
        prof = a + b * coord
        F[comp][...] = prof[:, None, None] if axis == 2 else prof[None, :, None]
        L = n[axis] * d[axis]
        for _ in range(25):
            pos = [rng.uniform(3 * d[0], (n[0] - 3) * d[0]), rng.uniform(0, n[1] * d[1]),
                   rng.uniform(0, n[2] * d[2])]
            pos[axis] = rng.uniform(3 * d[axis], L - 3 * d[axis])  # away from the seam
            out = orc.interp(c, F, pos)
            assert abs(out[comp] - (a + b * pos[axis])) < 1e-13, (comp, axis)
            assert max(abs(out[k]) for k in range(6) if k != comp) == 0.0


@pytest.mark.parametrize("window", [True, False])
def test_interp_3d_reproduces_fields_linear_in_all_axes(window):
    # f = a + bx x + by y + bz z on every component's own staggered nodes: the tensor
    # product of three quadratic splines reproduces it exactly, for each of the six
    # staggerings at once (a transposed axis or a wrong stagger bit fails here)
    n = (14, 12, 16)
    d = (0.15, 0.35, 0.2)
    c = orc.make_config(3, n, d, 0.05, window=window)
    shp = orc.field_shape(c)
    rng = np.random.default_rng(5 + window)
    coef = rng.uniform(-3, 3, (6, 4))
    F = []
    for comp in range(6):
        X = _stag_pos(n, d, comp, 0)[None, None, :]
        Y = _stag_pos(n, d, comp, 1)[None, :, None]
        Z = _stag_pos(n, d, comp, 2)[:, None, None]
        F.append(np.broadcast_to(coef[comp, 0] + coef[comp, 1] * X + coef[comp, 2] * Y
                                 + coef[comp, 3] * Z, shp).copy())
    for _ in range(40):
        pos = [rng.uniform(3 * d[a], (n[a] - 3) * d[a]) for a in range(3)]
        out = orc.interp(c, F, pos)
        want = coef[:, 0] + coef[:, 1:] @ np.array(pos)
        assert np.abs(out - want).max() < 1e-12


def test_interp_periodic_constant_and_y_linear():
    c = orc.make_config(2, (16, 16), (0.1, 0.2), 0.05)
    rng = np.random.default_rng(2)
    F = [np.full((16, 16), float(k + 1)) for k in range(6)]
    for _ in range(20):
        pos = [rng.uniform(0, 1.6), rng.uniform(0, 3.2)]
        assert np.allclose(orc.interp(c, F, pos), np.arange(1, 7), rtol=0, atol=1e-14)
    # linear in y, away from the periodic seam
    for comp in range(6):
        F = [np.zeros((16, 16)) for _ in range(6)]
        ypos = (np.arange(16) + 0.5 * STAG[comp][1]) * 0.2
        F[comp][...] = (1.0 + 3.0 * ypos)[:, None]
        for _ in range(10):
            pos = [rng.uniform(0, 1.6), rng.uniform(0.8, 2.2)]
            assert abs(orc.interp(c, F, pos)[comp] - (1.0 + 3.0 * pos[1])) < 1e-13


# ------------------------------------------------------------------ Esirkepov

def _div_j(c, J):
    """Backward-difference divergence of the staggered current on nodes."""
    dims = c.dims
    out = np.zeros(orc.field_shape(c))
    ax = {0: -1, 1: -2, 2: -3}  # numpy axis of x, y, z (last = x)
    for a in range(dims):
        out += (J[a] - np.roll(J[a], 1, axis=ax[a])) / c.d[a]
    return out


@pytest.mark.parametrize("dims", [2, 3])
def test_esirkepov_continuity_one_particle(dims):
    n = (12, 10, 8)[:dims]
    d = (0.1, 0.13, 0.11)[:dims]
    dt = 0.04
    c = orc.make_config(dims, n, d, dt)
    rng = np.random.default_rng(3 + dims)
    L = np.array(n) * np.array(d)
    for trial in range(60):
        p0 = rng.uniform(0, 1, dims) * L
        disp = rng.uniform(-0.99, 0.99, dims) * np.array(d) * (dt / min(d)) / (dt / min(d))
        if trial % 3 == 0:  # force cell crossings
            disp = np.sign(disp) * np.array(d) * rng.uniform(0.6, 0.99, dims)
        p1 = p0 + disp
        qw = rng.uniform(-2, 2)
        vz = rng.uniform(-0.5, 0.5)
        J = [np.zeros(orc.field_shape(c)) for _ in range(3)]
        orc.deposit(c, p0, p1, vz, qw, J)
        z0 = [p0[2]] if dims == 3 else None
        z1 = [p1[2]] if dims == 3 else None
        r0 = orc.rho(c, [p0[0]], [p0[1]], z0, [1.0], qw)
        # p1 may sit outside the box: rho wraps it periodically like the grid does
        r1 = orc.rho(c, [p1[0]], [p1[1]], z1, [1.0], qw)
        resid = (r1 - r0) / dt + _div_j(c, J)
        scale = abs(qw) / np.prod(d) / dt
        assert np.abs(resid).max() < 1e-13 * scale
        # total current: sum J dV = qw * velocity (2D: Jz uses vz)
        dV = np.prod(d)
        vel = disp / dt
        for a in range(dims):
            assert abs(J[a].sum() * dV - qw * vel[a]) < 1e-12 * abs(qw) * (abs(vel[a]) + 1)
        if dims == 2:
            assert abs(J[2].sum() * dV - qw * vz) < 1e-13 * (abs(qw) + 1)


@pytest.mark.parametrize("dims", [2, 3])
def test_esirkepov_at_rest_gives_zero_current(dims):
    n = (8, 8, 8)[:dims]
    d = (0.1, 0.1, 0.1)[:dims]
    c = orc.make_config(dims, n, d, 0.05)
    J = [np.zeros(orc.field_shape(c)) for _ in range(3)]
    p = [0.333, 0.471, 0.219][:dims]
    orc.deposit(c, p, p, 0.0, 1.7, J)
    assert all(np.abs(j).max() == 0.0 for j in J)


# ------------------------------------------------------------------ Yee

def _yee_run(c, E, B, nsteps):
    J = [np.zeros_like(E[0]) for _ in range(3)]
    hist = []
    for _ in range(nsteps):
        orc.yee_e(c, E, B, J)
        orc.yee_b(c, E, B)
        hist.append([e.copy() for e in E] + [b.copy() for b in B])
    return hist


def _predicted_cos(c, k):
    K2 = sum((2 * math.sin(k[a] * c.d[a] / 2) / c.d[a]) ** 2 for a in range(c.dims))
    return 1 - c.dt ** 2 * K2 / 2


@pytest.mark.parametrize("mode", ["TM", "TE"])
def test_yee_dispersion_2d(mode):
    n = (32, 24)
    d = (0.1, 0.15)
    dt = 0.9 / math.sqrt(1 / d[0] ** 2 + 1 / d[1] ** 2)
    c = orc.make_config(2, n, d, dt)
    k = (2 * math.pi * 3 / (n[0] * d[0]), 2 * math.pi * 2 / (n[1] * d[1]))
    E = [np.zeros((n[1], n[0])) for _ in range(3)]
    B = [np.zeros((n[1], n[0])) for _ in range(3)]
    X = np.arange(n[0])[None, :] * d[0]
    Y = np.arange(n[1])[:, None] * d[1]
    if mode == "TM":
        E[2][...] = np.cos(k[0] * X + k[1] * Y)  # Ez on nodes
        comp, arr = 2, "E"
    else:
        B[2][...] = np.cos(k[0] * (X + d[0] / 2) + k[1] * (Y + d[1] / 2))  # Bz
        comp, arr = 5, "B"
    hist = _yee_run(c, E, B, 40)
    series = np.array([h[comp] for h in hist])  # [t][y][x]
    cw = _predicted_cos(c, k)
    # single-mode leapfrog: F^{n+1} + F^{n-1} = 2 cos(omega dt) F^n at every point
    lhs = series[2:] + series[:-2]
    rhs = 2 * cw * series[1:-1]
    assert np.abs(lhs - rhs).max() < 1e-12
    # and the prediction is the Yee relation [sin(w dt/2)/dt]^2 = sum [sin(k d/2)/d]^2
    w = math.acos(cw) / dt
    lhs2 = (math.sin(w * dt / 2) / dt) ** 2
    rhs2 = sum((math.sin(k[a] * d[a] / 2) / d[a]) ** 2 for a in range(2))
    assert abs(lhs2 - rhs2) < 1e-12 * rhs2


def test_yee_dispersion_3d():
    n = (12, 10, 8)
    d = (0.1, 0.12, 0.14)
    dt = 0.9 / math.sqrt(sum(1 / x ** 2 for x in d))
    c = orc.make_config(3, n, d, dt)
    k = [2 * math.pi * m / (n[a] * d[a]) for a, m in enumerate((2, 1, 1))]
    shp = (n[2], n[1], n[0])
    E = [np.zeros(shp) for _ in range(3)]
    B = [np.zeros(shp) for _ in range(3)]
    Z, Y, X = np.meshgrid(np.arange(n[2]) * d[2], np.arange(n[1]) * d[1],
                          np.arange(n[0]) * d[0], indexing="ij")
    # start from B = discrete curl of A = (0, 0, Az): divergence-free on the Yee grid,
    # so the whole field is one transverse mode (no static part)
    Az = np.cos(k[0] * X + k[1] * Y + k[2] * (Z + d[2] / 2))  # on Ez positions
    B[0][...] = (np.roll(Az, -1, axis=1) - Az) / d[1]
    B[1][...] = -(np.roll(Az, -1, axis=2) - Az) / d[0]
    hist = _yee_run(c, E, B, 30)
    cw = _predicted_cos(c, k)
    for comp in (0, 1, 3, 4, 5):
        s = np.array([h[comp] for h in hist])
        assert np.abs(s[2:] + s[:-2] - 2 * cw * s[1:-1]).max() < 1e-12


def test_yee_magic_time_step_is_dispersion_free():
    # 1D (no y variation) at dt = dx: a right-moving wave shifts by exactly one cell
    nx, ny = 64, 4
    dx = 0.1
    c = orc.make_config(2, (nx, ny), (dx, 0.1), dx)  # building blocks do not check CFL
    X = np.arange(nx) * dx
    f = lambda x: np.exp(-((x - 3.2) / 0.4) ** 2)
    E = [np.zeros((ny, nx)) for _ in range(3)]
    B = [np.zeros((ny, nx)) for _ in range(3)]
    E[1][...] = f(X)[None, :]                    # Ey on (i, j+1/2) at t=0
    B[2][...] = f(X + dx / 2 - dx / 2)[None, :]  # Bz on (i+1/2) at t=+dt/2
    e0 = E[1][0].copy()
    for step in range(1, 11):
        orc.yee_e(c, E, B, [np.zeros((ny, nx))] * 3)
        orc.yee_b(c, E, B)
        assert np.abs(E[1][0] - np.roll(e0, step)).max() < 1e-13


# ------------------------------------------------------------------ full step invariants

def test_gauss_law_preserved_100_steps():
    w = inputs.thermal2d(nx=16, ny=16, d=0.1, uth=0.15, seed=7)
    p = w["params"]
    c = orc.make_config(2, p["n"][:2], p["d"][:2], p["dt"])
    s = orc.OracleSim(c, len(w["particles"]["x"]))
    s.set_particles(w["particles"])
    s.set_fields(w["E"], w["B"])
    s.set_rho_bg(None)
    g0 = s.gauss()
    rho_scale = 1.0  # n = 1
    assert np.abs(g0).max() < 1e-13
    for _ in range(10):
        s.step(10)
        g = s.gauss()
        assert np.abs(g - g0).max() < 1e-12 * rho_scale
    # and the plasma did evolve: fields are not zero
    f = s.get_fields()
    assert np.abs(f["Ex"]).max() > 1e-4


@pytest.mark.parametrize("dims", [2, 3])
def test_charge_density_moments(dims):
    """Charge density on the nodes from order-2 shapes: with E = 0 and no background,
    the Gauss residual is -rho. Its moments are fixed by the quadratic B-spline. The
    total is sum rho dV = q sum w. The first moment along x is q sum w x. The second is
    q sum w (x^2 + dx^2/4), since the spline's variance is a quarter cell. This holds
    for particles away from the periodic seam, where node positions do not wrap."""
    rng = np.random.default_rng(5 + dims)
    n = (16, 16, 8)[:dims]
    d = (0.1, 0.2, 0.15)[:dims]
    q_e = -1.0
    c = orc.make_config(dims, n, d, 0.01, q=q_e)
    N = 300
    L = [n[a] * d[a] for a in range(dims)]
    pos = [rng.uniform(0.3 * L[a], 0.7 * L[a], N) for a in range(dims)]
    p = dict(x=pos[0], y=pos[1], z=pos[2] if dims == 3 else np.zeros(N), ux=np.zeros(N),
             uy=np.zeros(N), uz=np.zeros(N), w=rng.uniform(0.5, 2.0, N),
             id=np.arange(N, dtype=np.int32))
    s = orc.OracleSim(c, N)
    s.set_particles(p)
    zero = np.zeros(n[::-1])
    s.set_fields([zero] * 3, [zero] * 3)
    s.set_rho_bg(zero)
    rho = -s.gauss()
    dV = float(np.prod(d))
    xn = np.arange(n[0]) * d[0]  # nodes along x (last array axis)
    tot = q_e * p["w"].sum()
    assert abs(rho.sum() * dV - tot) < 1e-12 * abs(tot)
    m1 = (rho * xn).sum() * dV
    assert abs(m1 - q_e * np.sum(p["w"] * p["x"])) < 1e-12 * abs(tot) * L[0]
    m2 = (rho * xn ** 2).sum() * dV
    want = q_e * np.sum(p["w"] * (p["x"] ** 2 + d[0] ** 2 / 4))
    assert abs(m2 - want) < 1e-12 * abs(tot) * L[0] ** 2


def test_energy_diagnostic_closed_forms():
    """Field energy (1/2) sum E^2 dV and B^2 alike, kinetic energy sum w m (gamma - 1),
    on states with closed-form values. One period of sin sampled at N >= 3 points sums
    its squares to N/2 exactly, so a unit sine in Ey holds V/4. A uniform Bz = 2 holds
    2 V. Momenta on Pythagorean triples give exact gamma: u = 3/4 gives 5/4, and
    u = 4/3 gives 5/3. The mass 2.5 catches a dropped m."""
    n, d = (16, 8), (0.1, 0.2)
    V = n[0] * d[0] * n[1] * d[1]
    c = orc.make_config(2, n, d, 0.05, m=2.5)
    s = orc.OracleSim(c, 8)
    x = np.arange(n[0])
    zero = np.zeros((n[1], n[0]))
    ey = np.repeat(np.sin(2 * np.pi * x / n[0])[None, :], n[1], 0)
    s.set_fields([zero, ey, zero], [zero, zero, np.full_like(zero, 2.0)])
    p = dict(x=np.array([0.3, 0.5, 0.7]), y=np.array([0.4, 0.4, 0.4]), z=np.zeros(3),
             ux=np.array([0.75, 0.0, 0.0]), uy=np.zeros(3), uz=np.array([0.0, 0.0, 4.0 / 3.0]),
             w=np.array([2.0, 5.0, 3.0]), id=np.arange(3, dtype=np.int32))
    s.set_particles(p)
    we, wb, wk = s.energy()
    assert abs(we - V / 4) < 1e-14 * V
    assert abs(wb - 2.0 * V) < 1e-14 * V
    assert abs(wk - 2.5 * (2.0 * 0.25 + 3.0 * 2.0 / 3.0)) < 1e-14


def _cold_plasma(dims, nx, d, side):
    """Cold electrons of density 1 on a side^dims lattice per cell of an nx x 4 (x 4)
    grid: positions, zero momenta, weights dV / ppc, ids."""
    n = (nx, 4, 4)[:dims]
    ax = [(np.arange(n[a])[:, None] + (np.arange(side) + 0.5)[None, :] / side).ravel() * d
          for a in range(dims)]
    pos = [g.ravel() for g in np.meshgrid(*ax, indexing="ij")]
    N = pos[0].size
    z = pos[2] if dims == 3 else np.zeros(N)
    return n, dict(x=pos[0], y=pos[1], z=z, ux=np.zeros(N), uy=np.zeros(N), uz=np.zeros(N),
                   w=np.full(N, d ** dims / side ** dims), id=np.arange(N, dtype=np.int32))


@pytest.mark.parametrize("dims", [2, 3])
def test_cold_plasma_oscillates_at_the_plasma_frequency(dims):
    """Full loop, closed form: a cold electron plasma of density 1 (q = -1, m = 1, so
    omega_p = 1) over a neutralising background starts with E = 0 and a small
    longitudinal velocity mode u_x = u0 sin(k x). It oscillates at the plasma frequency.
    The leapfrog makes that (2/dt) asin(omega_p dt/2), and the order-2 shapes lower it by
    a fraction of (k dx)^2, a few tenths of a percent at k dx = 0.1. Zero crossings of
    the mode's momentum over three periods give the frequency within 1 %. A wrong
    charge, mass, weight or current factor moves it much further: a factor 2 in the
    current would give sqrt(2)."""
    nx, d = 64, 0.1
    n, q = _cold_plasma(dims, nx, d, 4 if dims == 2 else 2)
    kx = 2.0 * math.pi / (nx * d)
    q["ux"] = 1e-3 * np.sin(kx * q["x"])
    dt = inputs.cfl_dt((d,) * dims)
    c = orc.make_config(dims, n, (d,) * dims, dt)
    s = orc.OracleSim(c, len(q["x"]))
    s.set_particles(q)
    zero = np.zeros(n[::-1])
    s.set_fields([zero] * 3, [zero] * 3)
    s.set_rho_bg(None)
    mode = []
    for _ in range(int(3 * 2 * math.pi / dt) + 5):
        s.step(1)
        r = s.get_particles()
        mode.append(float(np.sum(r["w"] * r["ux"] * np.sin(kx * r["x"]))))
    m = np.array(mode)
    # momenta live at half steps: m[j] is at t = (j + 1/2) dt
    t = (np.arange(len(m)) + 0.5) * dt
    i = np.nonzero(np.sign(m[:-1]) != np.sign(m[1:]))[0]
    zeros = t[i] - m[i] * (t[i + 1] - t[i]) / (m[i + 1] - m[i])
    assert len(zeros) >= 5
    omega = math.pi / np.mean(np.diff(zeros))
    want = 2.0 / dt * math.asin(dt / 2.0)
    assert abs(omega / want - 1.0) < 1e-2, (omega, want)
    assert omega < want  # the shapes' filtering lowers it


def test_gauss_law_preserved_3d():
    rng = np.random.default_rng(11)
    n, d = (8, 8, 8), (0.1, 0.1, 0.1)
    dt = 0.95 * 0.1 / math.sqrt(3)
    c = orc.make_config(3, n, d, dt)
    N = 2000
    p = dict(x=rng.uniform(0, 0.8, N), y=rng.uniform(0, 0.8, N), z=rng.uniform(0, 0.8, N),
             ux=rng.normal(0, 0.2, N), uy=rng.normal(0, 0.2, N), uz=rng.normal(0, 0.2, N),
             w=np.full(N, 0.512 / N), id=np.arange(N, dtype=np.int32))
    s = orc.OracleSim(c, N)
    s.set_particles(p)
    s.set_fields([np.zeros((8, 8, 8))] * 3, [np.zeros((8, 8, 8))] * 3)
    s.set_rho_bg(None)
    for _ in range(5):
        s.step(4)
        assert np.abs(s.gauss()).max() < 1e-12


def test_thermal_energy_drift_recorded():
    """Total energy drift of a small thermal plasma: recorded, loosely bounded
    (dx / lambda_D ~ 2.3 makes some grid heating expected)."""
    w = inputs.thermal2d(nx=32, ny=32, d=0.1, seed=9)
    p = w["params"]
    c = orc.make_config(2, p["n"][:2], p["d"][:2], p["dt"])
    s = orc.OracleSim(c, len(w["particles"]["x"]))
    s.set_particles(w["particles"])
    s.set_fields(w["E"], w["B"])
    e0 = s.energy().sum()
    s.step(100)
    e1 = s.energy().sum()
    assert np.isfinite(e1)
    assert abs(e1 - e0) / e0 < 0.1


# ------------------------------------------------------------------ moving window

def test_window_shift_translation_and_injection():
    w = inputs.lwfa2d(nx=64, ny=16, ppc=(2, 2), laser_back=4.0, ramp_cells=8)
    p = w["params"]
    c = orc.make_config(2, p["n"][:2], p["d"][:2], p["dt"], window=True, n0=p["n0"],
                        ramp_x0=p["ramp_x0"], ramp_len=p["ramp_len"],
                        inject_ppc=p["inject_ppc"])
    for n in range(0, 200, 7):
        assert orc.shift_count(c, n) == math.floor(n * p["dt"] / p["d"][0])
    # no particles, a field pattern, no current: fields after one shifting step equal
    # a field-only Yee step followed by a pure translation
    s = orc.OracleSim(c, 100000)
    s.set_particles({k: np.zeros(0) for k in orc.PARTICLE_KEYS} | {"id": np.zeros(0, np.int32)})
    s.set_fields(w["E"], w["B"])
    E = [e.copy() for e in w["E"]]
    B = [b.copy() for b in w["B"]]
    # dt/dx = 0.92: no shift after step 1, the first one after step 2
    for _ in range(2):
        orc.yee_e(c, E, B, [np.zeros_like(E[0])] * 3)
        orc.yee_b(c, E, B)
    s.step(1)
    assert s.shifts == 0
    s.step(1)
    assert orc.shift_count(c, 2) == 1 and s.shifts == 1
    f = s.get_fields()
    for a, k in enumerate(("Ex", "Ey", "Ez")):
        assert np.array_equal(f[k][:, :-1], E[a][:, 1:])
        assert np.all(f[k][:, -1] == 0)
    for a, k in enumerate(("Bx", "By", "Bz")):
        assert np.array_equal(f[k][:, :-1], B[a][:, 1:])
    # the uncovered column was filled with a cold 2x2 lattice at full density
    q = s.get_particles()
    assert len(q["x"]) == 16 * 4
    dx, dy = p["d"][0], p["d"][1]
    assert np.allclose(np.sort(np.unique(q["x"])), (63 + np.array([0.25, 0.75])) * dx)
    assert np.allclose(q["w"], p["n0"] * dx * dy / 4)
    assert np.all(q["ux"] == 0)


def test_window_drops_particles_leaving_left_edge():
    w = inputs.lwfa2d(nx=64, ny=16, ppc=(2, 2), laser_back=4.0, ramp_cells=8,
                      ramp_x0=-100.0, a0=0.0)
    p = w["params"]
    c = orc.make_config(2, p["n"][:2], p["d"][:2], p["dt"], window=True, n0=p["n0"],
                        ramp_x0=p["ramp_x0"], ramp_len=p["ramp_len"],
                        inject_ppc=p["inject_ppc"])
    s = orc.OracleSim(c, 100000)
    s.set_particles(w["particles"])
    s.set_fields(w["E"], w["B"])
    n0 = s.num_particles()
    assert n0 == 64 * 16 * 4
    s.step(2)  # one shift: the left column (x < dx) leaves, a new one enters
    q = s.get_particles()
    assert s.num_particles() == n0
    assert q["x"].min() >= 0.0
    assert q["id"].max() == n0 + 16 * 4 - 1


def test_window_3d_translation_injection_and_ids():
    """3D moving window: fields after a shifting step are a field-only Yee step then a
    pure translation; the uncovered x column (ny x nz cells) gets the injected lattice
    with the lab-frame weight; particles leaving x < 0 drop; ids continue from the
    largest one."""
    w = inputs.lwfa3d(nx=32, ny=8, nz=8, ppc=(2, 1, 2), laser_back=6.0, w0=3.0, tau=3.0,
                      ramp_cells=4, ramp_x0=-100.0, patch=(8, 8, 8))
    p = w["params"]
    c = orc.make_config(3, p["n"], p["d"], p["dt"], window=True, n0=p["n0"],
                        ramp_x0=p["ramp_x0"], ramp_len=p["ramp_len"], inject_ppc=p["inject_ppc"])
    dx = p["d"][0]
    steps = next(n for n in range(1, 10) if orc.shift_count(c, n) == 1)
    assert orc.shift_count(c, steps - 1) == 0 and steps == math.floor(dx / p["dt"]) + 1
    # fields: no particles
    s = orc.OracleSim(c, 100000)
    s.set_particles({k: np.zeros(0) for k in orc.PARTICLE_KEYS} | {"id": np.zeros(0, np.int32)})
    s.set_fields(w["E"], w["B"])
    E = [e.copy() for e in w["E"]]
    B = [b.copy() for b in w["B"]]
    for _ in range(steps):
        orc.yee_e(c, E, B, [np.zeros_like(E[0])] * 3)
        orc.yee_b(c, E, B)
    s.step(steps)
    assert s.shifts == 1
    f = s.get_fields()
    for a, k in enumerate(("Ex", "Ey", "Ez")):
        assert np.array_equal(f[k][:, :, :-1], E[a][:, :, 1:]) and np.all(f[k][:, :, -1] == 0)
    for a, k in enumerate(("Bx", "By", "Bz")):
        assert np.array_equal(f[k][:, :, :-1], B[a][:, :, 1:])
    q = s.get_particles()
    assert len(q["x"]) == 8 * 8 * 4  # ny * nz * (2 * 1 * 2)
    assert np.allclose(np.sort(np.unique(q["x"])), (31 + np.array([0.25, 0.75])) * dx)
    assert np.allclose(np.sort(np.unique(q["z"])), (np.arange(8)[:, None] + np.array([0.25, 0.75])).ravel() * p["d"][2])
    assert np.allclose(q["w"], p["n0"] * dx * p["d"][1] * p["d"][2] / 4)
    assert np.array_equal(np.sort(q["id"]), np.arange(len(q["x"])))
    # with plasma: the left column leaves, a new one enters, ids continue
    s2 = orc.OracleSim(c, 200000)
    s2.set_particles(w["particles"])
    s2.set_fields([np.zeros_like(e) for e in w["E"]], [np.zeros_like(b) for b in w["B"]])
    n0 = s2.num_particles()
    assert n0 == 32 * 8 * 8 * 4
    s2.step(steps)
    q2 = s2.get_particles()
    assert s2.num_particles() == n0 and q2["x"].min() >= 0.0
    assert q2["id"].max() == n0 + 8 * 8 * 4 - 1
