"""Patch decomposition across ranks with load-driven patch migration (Sec. 3.1, Figs. 3-4).

The paper's balancing method: the patches of the grid are ordered along a Hilbert
curve, each process owns a contiguous segment of that order, and the segments are
chosen from the patch loads (the SP count of a patch, Sec. 3) so that no process
carries much more than the average; when loads change, the segments are recomputed and
the patches whose owner changed move, fields and SP together. Between two rebalances,
each step exchanges the guard cells of the fields and the SP that crossed into patches
owned elsewhere.

This module holds that host-side machinery for several ranks, one per process:
  * Decomposition: the Hilbert order and the load-balanced segments (computed by the
    library's pic_hilbert_order and pic_partition), the owner of every patch and cell,
    and the migration plan between two ownerships;
  * exchange_particles: SP to the rank owning their patch (host-staged point-to-point);
  * exchange_guards / sum_guards: field values of owned cells to the ranks whose owned
    cells read them within a stencil width, and current deposited into cells owned
    elsewhere back to their owners (host-staged point-to-point).
Transfers go through torch.distributed send/recv of host tensors (gloo between CPU
processes); every rank derives the same index lists from the same ownership, so message
sizes need no negotiation beyond the particle counts.
"""
from __future__ import annotations

import numpy as np

from . import binding


class Decomposition:
    """Ownership of the patches of a grid of `ncells` cells in patches of `patch` cells
    (x fastest; 2D or 3D) by `nranks` ranks, from per-patch loads."""

    def __init__(self, dims: int, ncells, patch, nranks: int, periodic=(True, True, True)):
        self.dims = int(dims)
        self.n = tuple(int(v) for v in ncells[:dims])
        self.P = tuple(int(v) for v in patch[:dims])
        self.np = tuple(n // p for n, p in zip(self.n, self.P))
        self.npatch = int(np.prod(self.np))
        self.nranks = int(nranks)
        if not 1 <= self.nranks <= self.npatch:
            raise ValueError("need 1 <= ranks <= patches")
        self.periodic = tuple(bool(v) for v in periodic[:dims])
        self.order = binding.pic_hilbert_order(self.dims, self.np)
        self.owner = np.zeros(self.npatch, dtype=np.int32)
        self.max_load = 0.0

    # ---------------------------------------------------------------- ownership
    def partition(self, loads) -> np.ndarray:
        """Owner of every patch (index x fastest) from its load: contiguous Hilbert
        segments with the smallest largest segment load."""
        loads = np.asarray(loads, dtype=np.float64)
        first, mx = binding.pic_partition(loads[self.order], self.nranks)
        owner = np.empty(self.npatch, dtype=np.int32)
        for r in range(self.nranks):
            owner[self.order[first[r]:first[r + 1]]] = r
        self.owner = owner
        self.max_load = mx
        return owner

    def imbalance(self, loads) -> float:
        """Largest rank load over the mean rank load for the current owners."""
        loads = np.asarray(loads, dtype=np.float64)
        per = np.bincount(self.owner, weights=loads, minlength=self.nranks)
        return float(per.max() / max(per.mean(), 1e-300))

    def rebalance(self, loads, tolerance: float = 0.1):
        """Recomputes the segments when the current imbalance exceeds the best achievable
        one by more than `tolerance` (relative). Returns the migration plan (a list of
        (patch, from, to)), empty when nothing moves."""
        old = self.owner.copy()
        loads = np.asarray(loads, dtype=np.float64)
        current = np.bincount(old, weights=loads, minlength=self.nranks).max()
        new = self.partition(loads)
        if current <= (1.0 + tolerance) * self.max_load:
            self.owner = old
            return []
        return migration_plan(old, new)

    # ---------------------------------------------------------------- geometry
    def patch_of_cell(self) -> np.ndarray:
        """Patch index of every cell, in the field arrays' [nz][ny][nx] layout."""
        idx = [np.arange(n) // p for n, p in zip(self.n, self.P)]
        if self.dims == 2:
            return idx[0][None, :] + self.np[0] * idx[1][:, None]
        return (idx[0][None, None, :] + self.np[0] * idx[1][None, :, None]
                + self.np[0] * self.np[1] * idx[2][:, None, None])

    def owned_cells(self, rank: int) -> np.ndarray:
        """Boolean mask of the cells owned by `rank` ([nz][ny][nx] layout)."""
        return self.owner[self.patch_of_cell()] == rank

    def patch_of_positions(self, pos, d) -> np.ndarray:
        """Patch of each particle from its physical positions (list of arrays per axis)."""
        p = np.zeros(len(pos[0]), dtype=np.int64)
        mul = 1
        for a in range(self.dims):
            c = np.clip(np.floor(np.asarray(pos[a]) / d[a]).astype(np.int64), 0, self.n[a] - 1)
            p += (c // self.P[a]) * mul
            mul *= self.np[a]
        return p

    def dilate(self, mask: np.ndarray, width: int) -> np.ndarray:
        """Cells within `width` cells (per axis, a box) of the cells of `mask`, wrapping
        periodic axes and clipping the others."""
        out = mask.copy()
        axes = [mask.ndim - 1 - a for a in range(self.dims)]  # numpy axis of x, y, z
        for a, ax in enumerate(axes):
            cur = out.copy()
            for s in range(1, width + 1):
                for sgn in (1, -1):
                    sh = np.roll(out, sgn * s, axis=ax)
                    if not self.periodic[a]:
                        sl = [slice(None)] * mask.ndim
                        if sgn > 0:
                            sl[ax] = slice(0, s)
                        else:
                            sl[ax] = slice(-s, None)
                        sh[tuple(sl)] = False
                    cur |= sh
            out = cur
        return out

    def guard_lists(self, rank: int, width: int):
        """Flat indices of the cells this rank sends to (and receives from) every other
        rank in a guard exchange of `width` cells: to q, the cells owned here within
        `width` of a cell owned by q; from q, the cells owned by q within `width` of a
        cell owned here."""
        mine = self.owned_cells(rank)
        near_mine = self.dilate(mine, width)
        send, recv = {}, {}
        for q in range(self.nranks):
            if q == rank:
                continue
            theirs = self.owned_cells(q)
            s = np.flatnonzero((mine & self.dilate(theirs, width)).ravel())
            r = np.flatnonzero((theirs & near_mine).ravel())
            if len(s):
                send[q] = s
            if len(r):
                recv[q] = r
        return send, recv


def migration_plan(old_owner, new_owner):
    """(patch, from, to) for every patch whose owner changes, in patch order."""
    old_owner = np.asarray(old_owner)
    new_owner = np.asarray(new_owner)
    moved = np.flatnonzero(old_owner != new_owner)
    return [(int(p), int(old_owner[p]), int(new_owner[p])) for p in moved]


# -------------------------------------------------------------------- transfers
def _torch():
    import torch
    import torch.distributed as dist

    return torch, dist


def _exchange(send: dict, recv_sizes: dict, dtype, group=None):
    """Point-to-point exchange of 1D numpy arrays: send[q] goes to rank q; returns
    {q: array of recv_sizes[q] values} received from q. All sends are posted first."""
    torch, dist = _torch()
    reqs, out = [], {}
    for q, arr in sorted(send.items()):
        t = torch.from_numpy(np.ascontiguousarray(arr, dtype=dtype))
        reqs.append(dist.isend(t, dst=q, group=group))
    for q, n in sorted(recv_sizes.items()):
        t = torch.empty(int(n), dtype=torch.from_numpy(np.zeros(0, dtype=dtype)).dtype)
        dist.recv(t, src=q, group=group)
        out[q] = t.numpy()
    for r in reqs:
        r.wait()
    return out


def exchange_guards(field: np.ndarray, send_idx: dict, recv_idx: dict, group=None):
    """Writes into `field` the values of the cells other ranks own and this rank reads
    (host-staged): send_idx/recv_idx from Decomposition.guard_lists."""
    flat = field.reshape(-1)
    got = _exchange({q: flat[i] for q, i in send_idx.items()},
                    {q: len(i) for q, i in recv_idx.items()}, np.float64, group)
    for q, v in got.items():
        flat[recv_idx[q]] = v


def sum_guards(field: np.ndarray, owned: np.ndarray, send_idx: dict, recv_idx: dict,
               group=None):
    """Adds the contributions this rank deposited into cells owned by other ranks to
    those owners (the reverse of a guard exchange: send_idx here lists, per rank q, the
    cells q owns that this rank may have written, recv_idx the owned cells q may have
    written), then clears the cells this rank does not own."""
    flat = field.reshape(-1)
    got = _exchange({q: flat[i] for q, i in send_idx.items()},
                    {q: len(i) for q, i in recv_idx.items()}, np.float64, group)
    for q, v in sorted(got.items()):
        np.add.at(flat, recv_idx[q], v)
    flat[~owned.reshape(-1)] = 0.0


def exchange_particles(parts: dict, dest: np.ndarray, rank: int, group=None) -> dict:
    """Sends every particle whose destination rank differs from `rank` to that rank
    (host-staged: counts first, then each array) and returns this rank's particles:
    those it keeps, followed by the arrivals in source-rank order."""
    torch, dist = _torch()
    world = dist.get_world_size(group)
    keys = sorted(parts)
    dest = np.asarray(dest)
    counts = np.bincount(dest, minlength=world).astype(np.int64)
    # counts to every rank, counts from every rank
    send_counts = {q: np.array([counts[q]], np.int64) for q in range(world) if q != rank}
    got_counts = _exchange(send_counts, {q: 1 for q in range(world) if q != rank}, np.int64, group)
    keep = dest == rank
    out = {k: [np.asarray(parts[k])[keep]] for k in keys}
    for k in keys:
        arr = np.asarray(parts[k])
        dt = arr.dtype
        send = {q: arr[dest == q] for q in range(world) if q != rank and counts[q] > 0}
        recv = {q: int(got_counts[q][0]) for q in range(world)
                if q != rank and int(got_counts[q][0]) > 0}
        got = _exchange(send, recv, dt, group)
        for q in sorted(got):
            out[k].append(got[q])
    return {k: np.concatenate(v) for k, v in out.items()}
