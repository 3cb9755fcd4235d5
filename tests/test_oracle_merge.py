"""Pins of the oracle's particle merge (load limiting, Sec. 3.2), against what the
method must conserve and the choices it states; nothing here recomputes the merge.

* per group: total weight, momentum and energy kept to round-off, both new particles
  on the energy shell gamma = E/W, symmetric about P, coplanar with P and the
  smallest-id member's momentum, and carrying the two smallest ids;
* special cases: at rest, equal momenta (theta = 0), zero net momentum, < 3 members;
* over a sim: only overloaded patches change, groups never mix cells or momentum bins,
  per-cell totals are kept, survivors keep their positions, and the count drops by
  sum(N - 2) over the groups.
"""
import numpy as np
import pytest

import oracle as orc


@pytest.fixture(scope="module", autouse=True)
def built():
    orc.build()


def gam(u):
    return np.sqrt(1.0 + np.sum(np.asarray(u) ** 2, axis=0))


@pytest.mark.parametrize("n,scale,seed", [(3, 0.1, 1), (5, 1.0, 2), (17, 10.0, 3), (64, 0.01, 4)])
def test_group_conserves_and_is_symmetric(n, scale, seed):
    rng = np.random.default_rng(seed)
    u = rng.normal(0.3 * scale, scale, (3, n))
    w = rng.uniform(0.2, 2.0, n)
    ids = rng.permutation(10 * n)[:n].astype(np.int32)
    ua, ub, wn, (a, b) = orc.merge_group(u[0], u[1], u[2], w, ids)
    W, P, E = w.sum(), (w * u).sum(axis=1), (w * gam(u)).sum()
    assert abs(2 * wn - W) <= 1e-14 * W
    assert np.abs(wn * (ua + ub) - P).max() <= 1e-13 * (np.abs(w * u).sum(axis=1).max())
    assert abs(wn * (gam(ua) + gam(ub)) - E) <= 1e-13 * E
    assert abs(gam(ua) - E / W) <= 1e-13 * E / W and abs(gam(ub) - E / W) <= 1e-13 * E / W
    # symmetric about P: equal magnitudes, the difference normal to P
    assert abs(np.linalg.norm(ua) - np.linalg.norm(ub)) <= 1e-12 * np.linalg.norm(ua)
    assert abs(np.dot(ua - ub, P)) <= 1e-12 * np.linalg.norm(ua - ub) * np.linalg.norm(P)
    # coplanar with P and the reference (smallest-id) momentum
    ref = u[:, np.argmin(ids)]
    vol = np.dot(np.cross(ua, ub), ref)
    assert abs(vol) <= 1e-12 * np.linalg.norm(ua) * np.linalg.norm(ub) * np.linalg.norm(ref)
    assert sorted([ids[a], ids[b]]) == sorted(ids)[:2] and ids[a] < ids[b]


def test_group_special_cases():
    ids = np.array([7, 3, 9], dtype=np.int32)
    w = np.array([1.0, 2.0, 3.0])
    # at rest: both new particles at rest
    ua, ub, wn, _ = orc.merge_group(np.zeros(3), np.zeros(3), np.zeros(3), w, ids)
    assert np.all(ua == 0) and np.all(ub == 0) and wn == 3.0
    # equal momenta: theta = 0, both keep that momentum
    ux = np.full(3, 0.4)
    uy = np.full(3, -0.2)
    uz = np.full(3, 1.5)
    ua, ub, wn, _ = orc.merge_group(ux, uy, uz, w, ids)
    assert np.allclose(ua, [0.4, -0.2, 1.5], rtol=0, atol=1e-7)
    assert np.allclose(ub, [0.4, -0.2, 1.5], rtol=0, atol=1e-7)
    # zero net momentum: u_a = -u_b with gamma = E/W
    ux = np.array([1.0, -0.5, 0.0])
    w0 = np.array([1.0, 2.0, 5.0])
    ua, ub, wn, (a, b) = orc.merge_group(ux, np.zeros(3), np.zeros(3), w0, ids)
    assert np.allclose(ua, -ub, atol=1e-15)
    E = (w0 * gam(np.vstack([ux, np.zeros(3), np.zeros(3)]))).sum()
    assert abs(gam(ua) - E / w0.sum()) < 1e-14
    # fewer than three members: nothing to merge
    assert orc.merge_group([0.1, 0.2], [0.0, 0.0], [0.0, 0.0], [1.0, 1.0],
                           np.array([1, 2], dtype=np.int32)) is None


def _sim_with_hot_patch(seed=5):
    """16x16 periodic grid in 8x8 patches; patch 0 holds 600 particles in 3 cells with
    clustered momenta, the rest 4 per cell with thermal momenta."""
    rng = np.random.default_rng(seed)
    d = 0.1
    c = orc.make_config(2, (16, 16), (d, d), 0.05)
    xs, ys, us = [], [], []
    for (ci, cj) in ((1, 1), (2, 1), (5, 6)):
        m = 200
        xs.append((ci + rng.random(m)) * d)
        ys.append((cj + rng.random(m)) * d)
        us.append(rng.normal([[0.5], [0.0], [0.0]], 0.08, (3, m)))
    for i in range(16):
        for j in range(16):
            if i < 8 and j < 8:
                continue
            xs.append((i + rng.random(4)) * d)
            ys.append((j + rng.random(4)) * d)
            us.append(rng.normal(0.0, 0.05, (3, 4)))
    x, y, u = np.concatenate(xs), np.concatenate(ys), np.concatenate(us, axis=1)
    n = len(x)
    p = dict(x=x, y=y, z=np.zeros(n), ux=u[0], uy=u[1], uz=u[2],
             w=rng.uniform(0.5, 1.5, n), id=rng.permutation(n).astype(np.int32))
    o = orc.OracleSim(c, n)
    o.set_particles(p)
    return c, o, p


def _totals_by_cell(p, d=0.1, nx=16):
    cell = (np.floor(p["y"] / d) * nx + np.floor(p["x"] / d)).astype(int)
    u = np.vstack([p["ux"], p["uy"], p["uz"]])
    out = {}
    for c in np.unique(cell):
        k = cell == c
        out[c] = (p["w"][k].sum(), (p["w"][k] * u[:, k]).sum(axis=1), (p["w"][k] * gam(u[:, k])).sum())
    return out


def test_sim_merge_conserves_per_cell_and_limits_the_hot_patch():
    c, o, p0 = _sim_with_hot_patch()
    removed = o.merge((8, 8), above=400, dp=0.1)
    p1 = o.get_particles()
    assert removed > 0 and o.num_particles() == len(p0["x"]) - removed
    # survivors are original particles at their original positions
    i0 = np.argsort(p0["id"])
    assert np.all(np.isin(p1["id"], p0["id"]))
    pos = np.searchsorted(p0["id"][i0], p1["id"])
    assert np.array_equal(p1["x"], p0["x"][i0][pos]) and np.array_equal(p1["y"], p0["y"][i0][pos])
    # particles outside the overloaded patch are untouched
    hot0 = (p0["x"] < 0.8) & (p0["y"] < 0.8)
    cold_ids = np.sort(p0["id"][~hot0])
    k1 = np.isin(p1["id"], cold_ids)
    assert k1.sum() == len(cold_ids)
    for key in ("ux", "uy", "uz", "w"):
        a = p1[key][k1]
        b = p0[key][i0][pos][k1]
        assert np.array_equal(a, b)
    # per-cell totals of weight, momentum and energy are kept
    t0, t1 = _totals_by_cell(p0), _totals_by_cell(p1)
    assert t0.keys() == t1.keys()
    for cc in t0:
        assert abs(t1[cc][0] - t0[cc][0]) <= 1e-13 * t0[cc][0]
        assert np.abs(t1[cc][1] - t0[cc][1]).max() <= 1e-12 * max(1.0, np.abs(t0[cc][1]).max())
        assert abs(t1[cc][2] - t0[cc][2]) <= 1e-13 * t0[cc][2]
    # the count drop is sum(N - 2) over groups of >= 3 in (cell, momentum bin)
    u0 = np.vstack([p0["ux"], p0["uy"], p0["uz"]])
    keys = {}
    for k in np.nonzero(hot0)[0]:
        kk = (int(p0["x"][k] // 0.1), int(p0["y"][k] // 0.1)) + tuple(int(v) for v in np.floor(u0[:, k] / 0.1))
        keys[kk] = keys.get(kk, 0) + 1
    assert removed == sum(m - 2 for m in keys.values() if m >= 3)


def test_sim_merge_below_threshold_changes_nothing():
    c, o, p0 = _sim_with_hot_patch(seed=6)
    assert o.merge((8, 8), above=100000, dp=0.1) == 0
    p1 = o.get_particles()
    i0 = np.argsort(p0["id"])
    for key in ("x", "y", "ux", "uy", "uz", "w"):
        assert np.array_equal(p1[key], p0[key][i0])


def test_sim_merge_hysteresis():
    """A patch merged once is not merged again until it grows past 5/4 of its count
    after that pass, even while it stays above the threshold."""
    c, o, p0 = _sim_with_hot_patch(seed=7)
    first = o.merge((8, 8), above=200, dp=0.1)
    n1 = o.num_particles()
    hot = (o.get_particles()["x"] < 0.8) & (o.get_particles()["y"] < 0.8)
    assert first > 0 and hot.sum() > 200  # still above the threshold
    assert o.merge((8, 8), above=200, dp=0.1) == 0 and o.num_particles() == n1
    # a fresh particle set clears the memory: the same merge happens again
    o.set_particles(p0)
    assert o.merge((8, 8), above=200, dp=0.1) == first
