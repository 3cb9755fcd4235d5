"""Pins of the oracle's particle splitting (load limiting in low-density cells, Sec. 3.2)
against what the conservation laws and the stated rule fix, with no GPU:
  * per split: total weight, momentum sum w u and kinetic energy sum w (gamma - 1) kept;
    the charge centroid kept; the second moment of the charge density raised by exactly
    q w delta^2 per axis (the spline's own variance is unchanged), checked through the
    oracle's charge density, an independent code path;
  * both halves in the parent's cell;
  * the count rise equals sum over cells with 1 <= n < below of min(eligible, below - n),
    counted here by brute force from the positions and weights;
  * which particles split (smallest ids first), the weight floor, untouched cells;
  * new ids: next id + rank in (patch, cell, parent id) order.
"""
import math

import numpy as np
import pytest

import oracle as orc


def _sim(dims, n, d, parts, window=False):
    c = orc.make_config(dims, n[:dims], d[:dims], 0.5 * min(d[:dims]), window=window)
    o = orc.OracleSim(c, 4 * len(parts["x"]) + 64)
    o.set_particles(parts)
    z = np.zeros(orc.field_shape(c))
    o.set_fields([z, z, z], [z, z, z])
    return c, o


def _parts(x, y, z=None, w=None, u=None, ids=None):
    m = len(x)
    rng = np.random.default_rng(3)
    u = rng.normal(0, 0.3, (3, m)) if u is None else u
    return dict(x=np.asarray(x, float), y=np.asarray(y, float),
                z=np.zeros(m) if z is None else np.asarray(z, float), ux=u[0], uy=u[1], uz=u[2],
                w=np.ones(m) if w is None else np.asarray(w, float),
                id=np.arange(m, dtype=np.int32) if ids is None else np.asarray(ids, np.int32))


def _totals(p):
    g = np.sqrt(1 + p["ux"] ** 2 + p["uy"] ** 2 + p["uz"] ** 2)
    w = p["w"]
    return np.array([w.sum(), (w * p["ux"]).sum(), (w * p["uy"]).sum(), (w * p["uz"]).sum(),
                     (w * (g - 1)).sum(), (w * p["x"]).sum(), (w * p["y"]).sum(),
                     (w * p["z"]).sum()])


@pytest.mark.parametrize("dims", [2, 3])
def test_one_split_conserves_and_moves_the_second_moment(dims):
    n, d = (8, 8, 8), (0.3, 0.2, 0.25)
    x, y, z = [0.3 * 3 + 0.07], [0.2 * 5 + 0.15], [0.25 * 2 + 0.05]
    p = _parts(x, y, z if dims == 3 else None, w=[0.8])
    c, o = _sim(dims, n, d, p)
    rho0 = orc.rho(c, p["x"], p["y"], p["z"], p["w"], -1.0)
    k = o.split((4, 4, 4)[:dims], below=4, wmin=0.1)
    assert k == 1 and o.num_particles() == 2
    q = o.get_particles()
    assert np.allclose(_totals(q), _totals(p), rtol=0, atol=1e-15)
    assert np.all(q["w"] == 0.4)
    for key in ("ux", "uy", "uz"):
        assert q[key][0] == q[key][1] == p[key][0]
    # both halves in the parent's cell, symmetric about it
    for a, key in enumerate(("x", "y", "z")[:dims]):
        cells = np.floor(q[key] / d[a])
        assert np.all(cells == math.floor(p[key][0] / d[a]))
    # second moment of the charge density through orc_rho: +q w delta_a^2 per axis
    rho1 = orc.rho(c, q["x"], q["y"], q["z"], q["w"], -1.0)
    dV = np.prod(d[:dims])
    shp = orc.field_shape(c)
    grids = np.meshgrid(*[np.arange(n[a]) * d[a] for a in range(dims)][::-1], indexing="ij")[::-1]
    for a, key in enumerate(("x", "y", "z")[:dims]):
        f = p[key][0] / d[a] - math.floor(p[key][0] / d[a])
        delta = 0.5 * min(f, 1 - f) * d[a]
        X = grids[a].reshape(shp)
        m1 = ((rho1 - rho0) * X).sum() * dV
        m2 = ((rho1 - rho0) * X * X).sum() * dV
        assert abs(m1) < 1e-12
        assert abs(m2 - (-1.0) * 0.8 * delta ** 2) < 1e-12


def test_which_particles_split_and_their_ids():
    # one 4x4 patch per quadrant of an 8x8 grid (patch 4x4): cell counts 1, 2, 3, 4, 5
    d = (0.5, 0.5)
    cell = lambda i, j, fx=0.3, fy=0.6: ((i + fx) * d[0], (j + fy) * d[1])
    pts, ids, ws = [], [], []
    # patch 0 (cells x<4, y<4): cell (1,1) holds 3 particles (ids 30, 10, 20); cell (2,0) 1
    for i, pid in enumerate((30, 10, 20)):
        pts.append(cell(1, 1, 0.2 + 0.2 * i)); ids.append(pid); ws.append(1.0)
    pts.append(cell(2, 0)); ids.append(5); ws.append(1.0)
    # patch 1 (x>=4, y<4): cell (5,2) holds 4 particles -> untouched at below = 4
    for i in range(4):
        pts.append(cell(5, 2, 0.1 + 0.2 * i)); ids.append(40 + i); ws.append(1.0)
    # patch 2 (x<4, y>=4): cell (0,6): 2 particles, one below the weight floor
    pts.append(cell(0, 6, 0.4)); ids.append(7); ws.append(0.15)
    pts.append(cell(0, 6, 0.8)); ids.append(8); ws.append(0.5)
    x, y = zip(*pts)
    p = _parts(x, y, w=ws, ids=ids)
    c, o = _sim(2, (8, 8, 1), d, p)
    k = o.split((4, 4), below=4, wmin=0.1)
    # patch 0: cell (2,0) [local index 2] before cell (1,1) [local index 5]:
    #   (2,0): 1 particle, room 3, one eligible -> 1 split (id 5 -> child next_id + 0)
    #   (1,1): 3 particles, room 1 -> the smallest id (10) splits -> child next_id + 1
    # patch 1: none (4 particles). patch 2: cell (0,6): id 7 below the floor (0.15 < 0.2),
    #   id 8 splits -> child next_id + 2
    assert k == 3
    q = o.get_particles()
    nid = max(ids) + 1
    assert list(q["id"][-3:]) == [nid, nid + 1, nid + 2]
    byid = {int(i): j for j, i in enumerate(q["id"])}
    assert q["w"][byid[5]] == 0.5 and q["w"][byid[nid]] == 0.5
    assert q["w"][byid[10]] == 0.5 and q["w"][byid[nid + 1]] == 0.5
    assert q["w"][byid[20]] == 1.0 and q["w"][byid[30]] == 1.0
    assert q["w"][byid[7]] == 0.15 and q["w"][byid[8]] == 0.25 and q["w"][byid[nid + 2]] == 0.25
    for i in range(4):
        assert q["w"][byid[40 + i]] == 1.0
    # a second pass: (2,0) now holds 2 -> both split; (1,1) holds 4 -> none; (0,6) holds 3
    # (id 7 ineligible, id 8 and its child at 0.25 >= 0.2 eligible, room 1) -> id 8
    assert o.split((4, 4), below=4, wmin=0.1) == 3


@pytest.mark.parametrize("dims", [2, 3])
def test_count_rise_matches_brute_force_on_a_sparse_plasma(dims):
    rng = np.random.default_rng(17 + dims)
    n = (16, 8, 8) if dims == 3 else (32, 16, 1)
    d = (0.1, 0.15, 0.2)
    m = int(0.8 * np.prod(n[:dims]))  # under one particle per cell on average
    pos = [rng.uniform(0, n[a] * d[a], m) for a in range(dims)]
    w = rng.choice([0.05, 0.3, 1.0], m)
    p = _parts(pos[0], pos[1], pos[2] if dims == 3 else None, w=w,
               ids=rng.permutation(m).astype(np.int32))
    c, o = _sim(dims, n, d, p)
    below, wmin = 3, 0.1
    # brute force: counts and eligible particles per cell
    cells = np.zeros(m, dtype=np.int64)
    mul = 1
    for a in range(dims):
        cells += np.clip(np.floor(pos[a] / d[a]).astype(np.int64), 0, n[a] - 1) * mul
        mul *= n[a]
    cnt = np.bincount(cells, minlength=mul)
    elig = np.bincount(cells[w >= 2 * wmin], minlength=mul)
    want = int(sum(min(e, below - k) for k, e in zip(cnt, elig) if 1 <= k < below))
    t0 = _totals(p)
    k = o.split((8, 8, 8)[:dims] if dims == 3 else (8, 8), below=below, wmin=wmin)
    assert k == want and o.num_particles() == m + want
    q = o.get_particles()
    assert np.abs(_totals(q) - t0).max() < 1e-12 * np.abs(t0).max()
    assert len(np.unique(q["id"])) == len(q["id"])


def test_window_positions_stay_inside_the_window():
    # a particle in the last cell of a window keeps both halves inside [0, Lx)
    d = (0.125, 0.5)
    p = _parts([64 * 0.125 - 1e-3, 0.01], [1.0, 1.0], w=[1.0, 1.0])
    c, o = _sim(2, (64, 8, 1), d, p, window=True)
    assert o.split((16, 8), below=2, wmin=0.1) == 2
    q = o.get_particles()
    assert q["x"].min() >= 0.0 and q["x"].max() < 64 * 0.125
