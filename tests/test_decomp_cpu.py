"""Patch decomposition across ranks (Sec. 3.1, Figs. 3-4), host side, no GPU:

* the Hilbert order is a permutation whose consecutive patches are face neighbours on
  square power-of-two grids (2D and 3D), and stays a permutation on other grids;
* the partition is the optimal contiguous one (checked against a brute-force dynamic
  program on small inputs), every rank owning at least one patch;
* rebalancing moves exactly the patches whose owner changed, and only beyond its
  tolerance; guard lists agree between sender and receiver;
* on two and four gloo ranks, a small periodic PIC run split over Hilbert segments
  (host-staged guard exchange of E and B, current summed back to the owners, particles
  sent to the owner of their patch, one rebalance with migration half way) gives the
  single-rank oracle run's fields and particles to 1e-12. The per-rank PIC arithmetic
  is the oracle's building blocks (interpolation, Boris, Esirkepov, Yee): the test
  drives the decomposition module with it.
"""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle as orc  # noqa: E402
from paper_1511_03878_gb300 import binding, decomp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _neighbours(a, b, np_):
    ca = np.unravel_index(a, np_[::-1])
    cb = np.unravel_index(b, np_[::-1])
    return sum(abs(int(x) - int(y)) for x, y in zip(ca, cb)) == 1


@pytest.mark.parametrize("dims,np_", [(2, (8, 8)), (2, (16, 16)), (3, (4, 4, 4)), (3, (8, 8, 8))])
def test_hilbert_order_walks_face_neighbours(dims, np_):
    o = binding.pic_hilbert_order(dims, np_)
    assert sorted(o.tolist()) == list(range(int(np.prod(np_))))
    assert all(_neighbours(int(a), int(b), np_) for a, b in zip(o[:-1], o[1:]))


@pytest.mark.parametrize("dims,np_", [(2, (8, 4)), (2, (6, 5)), (3, (5, 3, 2)), (3, (1, 7, 3))])
def test_hilbert_order_on_other_grids_is_a_permutation(dims, np_):
    o = binding.pic_hilbert_order(dims, np_)
    assert sorted(o.tolist()) == list(range(int(np.prod(np_))))


def _best_minmax(load, k):
    """Optimal largest segment load of a contiguous split into k non-empty segments."""
    n = len(load)
    pre = np.concatenate([[0.0], np.cumsum(load)])
    INF = float("inf")
    f = [[INF] * (n + 1) for _ in range(k + 1)]
    f[0][0] = 0.0
    for j in range(1, k + 1):
        for i in range(1, n + 1):
            for m in range(j - 1, i):
                f[j][i] = min(f[j][i], max(f[j - 1][m], pre[i] - pre[m]))
    return f[k][n]


def test_partition_is_optimal_and_contiguous():
    rng = np.random.default_rng(7)
    for trial in range(60):
        n = int(rng.integers(1, 12))
        k = int(rng.integers(1, n + 1))
        load = rng.lognormal(0, 1.5, n) if trial % 3 else rng.integers(0, 5, n).astype(float)
        first, mx = binding.pic_partition(load, k)
        assert first[0] == 0 and first[-1] == n
        assert np.all(np.diff(first) >= 1)  # every rank owns a patch
        seg = [load[first[r]:first[r + 1]].sum() for r in range(k)]
        assert abs(max(seg) - mx) <= 1e-12 * max(1.0, mx)
        assert mx <= _best_minmax(load, k) * (1 + 1e-9) + 1e-12


def test_partition_rejects_bad_input():
    with pytest.raises(binding.PicError):
        binding.pic_partition([1.0, 2.0], 3)
    with pytest.raises(binding.PicError):
        binding.pic_partition([1.0, -2.0], 1)
    with pytest.raises(binding.PicError):
        binding.pic_partition([1.0, float("nan")], 1)


def test_rebalance_moves_only_changed_patches():
    d = decomp.Decomposition(2, (64, 32), (8, 8), 4)
    flat = np.full(d.npatch, 100.0)
    d.partition(flat)
    assert d.imbalance(flat) == pytest.approx(1.0)
    assert d.rebalance(flat, tolerance=0.05) == []  # already balanced
    heavy = flat.copy()
    heavy[d.order[:4]] = 1000.0  # the first patches along the curve become heavy
    old = d.owner.copy()
    plan = d.rebalance(heavy, tolerance=0.05)
    assert plan and d.imbalance(heavy) < 1.3
    changed = np.flatnonzero(old != d.owner)
    assert [p for p, _, _ in plan] == changed.tolist()
    for p, a, b in plan:
        assert old[p] == a and d.owner[p] == b


def test_guard_lists_agree_between_ranks():
    d = decomp.Decomposition(2, (32, 16), (8, 8), 3)
    rng = np.random.default_rng(2)
    d.partition(rng.uniform(1, 10, d.npatch))
    lists = [d.guard_lists(r, 2) for r in range(3)]
    for r in range(3):
        send, recv = lists[r]
        for q, idx in send.items():
            assert np.array_equal(idx, lists[q][1][r])
        owned = d.owned_cells(r).ravel()
        for q, idx in recv.items():
            assert not owned[idx].any()


# ------------------------------------------------------------------ distributed run

N, D, P, DT = (32, 16), (0.1, 0.15), (8, 8), 0.05
KEYS = ("x", "y", "z", "ux", "uy", "uz", "w")


def _initial():
    """A periodic 2D plasma with a dense blob (uneven patch loads) and small random
    initial fields."""
    rng = np.random.default_rng(11)
    m0, m1 = 250, 350
    x = np.concatenate([rng.uniform(0, N[0] * D[0], m0), rng.normal(0.8, 0.25, m1) % (N[0] * D[0])])
    y = np.concatenate([rng.uniform(0, N[1] * D[1], m0), rng.normal(1.2, 0.3, m1) % (N[1] * D[1])])
    m = m0 + m1
    parts = dict(x=x, y=y, z=np.zeros(m), ux=rng.normal(0, 0.1, m), uy=rng.normal(0, 0.1, m),
                 uz=rng.normal(0, 0.1, m), w=rng.uniform(0.5, 1.5, m) * 0.01,
                 id=np.arange(m, dtype=np.int32))
    shp = (N[1], N[0])
    E = [rng.normal(0, 0.01, shp) for _ in range(3)]
    B = [rng.normal(0, 0.01, shp) for _ in range(3)]
    return parts, E, B


def _config():
    return orc.make_config(2, N, D, DT)


def _single_rank(steps):
    parts, E, B = _initial()
    o = orc.OracleSim(_config(), 4 * len(parts["x"]))
    o.set_particles(parts)
    o.set_fields(E, B)
    o.step(steps)
    return o.get_particles(), o.get_fields()


def _local_step(c, parts, E, Bh, Bn, dec, rank, lists):
    """One PIC step of this rank's particles (oracle building blocks), then the guard
    and particle exchanges of the decomposition."""
    J = [np.zeros((N[1], N[0])) for _ in range(3)]
    F = [E[0], E[1], E[2], Bn[0], Bn[1], Bn[2]]
    L = (N[0] * D[0], N[1] * D[1])
    for i in range(len(parts["x"])):
        pos0 = [parts["x"][i], parts["y"][i]]
        eb = orc.interp(c, F, pos0)
        u = orc.boris(c.q, c.m, c.dt, eb[:3], eb[3:], [parts["ux"][i], parts["uy"][i], parts["uz"][i]])
        g = np.sqrt(1.0 + u @ u)
        pos1 = [pos0[0] + c.dt * u[0] / g, pos0[1] + c.dt * u[1] / g]
        orc.deposit(c, pos0, pos1, u[2] / g, c.q * parts["w"][i], J)
        parts["x"][i] = pos1[0] % L[0] if pos1[0] < 0 or pos1[0] >= L[0] else pos1[0]
        parts["y"][i] = pos1[1] % L[1] if pos1[1] < 0 or pos1[1] >= L[1] else pos1[1]
        parts["ux"][i], parts["uy"][i], parts["uz"][i] = u
    owned = dec.owned_cells(rank)
    s3, r3 = lists[3]
    for a in range(3):  # current deposited into cells owned elsewhere -> their owners
        decomp.sum_guards(J[a], owned, r3, s3)
    orc.yee_e(c, E, Bh, J)
    s2, r2 = lists[2]
    for a in range(3):
        decomp.exchange_guards(E[a], s2, r2)
    Bold = [b.copy() for b in Bh]
    orc.yee_b(c, E, Bh)
    for a in range(3):
        decomp.exchange_guards(Bh[a], s2, r2)
    for a in range(3):
        Bn[a][...] = 0.5 * (Bold[a] + Bh[a])
    dest = dec.owner[dec.patch_of_positions([parts["x"], parts["y"]], D)]
    return decomp.exchange_particles(parts, dest, rank)


def _rank_main(rank, world, port, q, steps_before, steps_after):
    import sys

    sys.path.insert(0, ROOT)
    import torch.distributed as dist

    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank,
                            world_size=world)
    try:
        c = _config()
        parts0, E, B = _initial()
        dec = decomp.Decomposition(2, N, P, world)
        counts = np.bincount(dec.patch_of_positions([parts0["x"], parts0["y"]], D),
                             minlength=dec.npatch)
        dec.partition(np.ones(dec.npatch))  # start from an even split by patch count
        mine = dec.owner[dec.patch_of_positions([parts0["x"], parts0["y"]], D)] == rank
        parts = {k: np.array(v[mine]) for k, v in parts0.items()}
        Bh = [b.copy() for b in B]
        Bn = [b.copy() for b in B]
        lists = {2: dec.guard_lists(rank, 2), 3: dec.guard_lists(rank, 3)}
        for _ in range(steps_before):
            parts = _local_step(c, parts, E, Bh, Bn, dec, rank, lists)
        # rebalance on the SP counts (all ranks see the same counts), migrate patches:
        # the particles of a patch that changes owner go with it; every rank holds the
        # replicated fields' guard and owned cells of its new segment after one exchange
        mycount = np.bincount(dec.patch_of_positions([parts["x"], parts["y"]], D),
                              minlength=dec.npatch).astype(np.float64)
        t = torch.from_numpy(mycount)
        dist.all_reduce(t)
        counts = t.numpy()
        old_owner = dec.owner.copy()
        plan = dec.rebalance(counts, tolerance=0.0)
        moved = len(plan)
        if plan:
            # fields of migrating patches: their old owners send them (a patch's cells
            # are a guard-free block, so an owner-to-owner copy of the block suffices)
            pc = dec.patch_of_cell()
            for arrs in (E, Bh, Bn):
                for a in range(3):
                    send = {}
                    recv = {}
                    for p, src, dst in plan:
                        cells = np.flatnonzero((pc == p).ravel())
                        if src == rank:
                            send.setdefault(dst, []).append(cells)
                        if dst == rank:
                            recv.setdefault(src, []).append(cells)
                    send = {k: np.concatenate(v) for k, v in send.items()}
                    recv = {k: np.concatenate(v) for k, v in recv.items()}
                    flat = arrs[a].reshape(-1)
                    got = decomp._exchange({k: flat[v] for k, v in send.items()},
                                           {k: len(v) for k, v in recv.items()}, np.float64)
                    for k, v in got.items():
                        flat[recv[k]] = v
            dest = dec.owner[dec.patch_of_positions([parts["x"], parts["y"]], D)]
            parts = decomp.exchange_particles(parts, dest, rank)
            lists = {2: dec.guard_lists(rank, 2), 3: dec.guard_lists(rank, 3)}
            s2, r2 = lists[2]
            for arrs in (E, Bh, Bn):
                for a in range(3):
                    decomp.exchange_guards(arrs[a], s2, r2)
        for _ in range(steps_after):
            parts = _local_step(c, parts, E, Bh, Bn, dec, rank, lists)
        owned = dec.owned_cells(rank)
        fields = {k: np.where(owned, v, np.nan) for k, v in
                  zip(("Ex", "Ey", "Ez", "Bx", "By", "Bz", "Bnx", "Bny", "Bnz"), E + Bh + Bn)}
        q.put((rank, parts, fields, moved, bool((old_owner != dec.owner).any())))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 4])
def test_distributed_run_matches_single_rank(world):
    steps_before, steps_after = 3, 3
    ctx = torch.multiprocessing.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, q, steps_before, steps_after))
             for r in range(world)]
    for p in procs:
        p.start()
    results = [q.get(timeout=300) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
    assert all(p.exitcode == 0 for p in procs), [p.exitcode for p in procs]
    qo, fo = _single_rank(steps_before + steps_after)
    # particles: the union over ranks, matched by id
    parts = {k: np.concatenate([r[1][k] for r in results]) for k in KEYS + ("id",)}
    order = np.argsort(parts["id"])
    parts = {k: v[order] for k, v in parts.items()}
    assert np.array_equal(parts["id"], qo["id"])
    for k in ("ux", "uy", "uz", "w"):
        assert np.abs(parts[k] - qo[k]).max() <= 1e-12 * np.abs(qo[k]).max(), k
    for k, L in (("x", N[0] * D[0]), ("y", N[1] * D[1])):
        dd = (parts[k] - qo[k] + 0.5 * L) % L - 0.5 * L
        assert np.abs(dd).max() <= 1e-12 * L, k
    # fields: every cell from its owner
    assert any(r[3] > 0 for r in results)  # the rebalance migrated patches
    for k in ("Ex", "Ey", "Ez", "Bx", "By", "Bz", "Bnx", "Bny", "Bnz"):
        full = np.full(fo[k].shape, np.nan)
        for r in results:
            m = ~np.isnan(r[2][k])
            full[m] = r[2][k][m]
        assert not np.isnan(full).any()
        assert np.abs(full - fo[k]).max() <= 1e-12 * np.abs(fo[k]).max(), k


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]
