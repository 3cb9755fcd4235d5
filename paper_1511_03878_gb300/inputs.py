"""Seeded synthetic inputs (initial conditions) shaped like the paper's workloads.

This module holds no step of the PIC method: it only draws particle lattices,
momenta and laser fields. It is the one piece that serves both the CUDA path and
the CPU oracle, so it imports neither.

Workloads (normalised units, c = 1, electrons q = -1, m = 1):
  * thermal2d  - 2D3V periodic thermal plasma, 4x4 quiet lattice per cell, Gaussian
                 momenta (u_th = 0.044, about 1 keV), n = 1 (omega_p = 1).
  * lwfa2d     - 2D3V laser-wakefield run in a moving window: a cold 2x2 lattice of
                 electrons over a linear density ramp and a linearly polarised
                 Gaussian pulse, shaped like the CILEX "F2" case of Sec. 2.2 (laser
                 focused at the foot of the ramp, duration given as FWHM in
                 intensity, Gaussian in all directions) scaled to 2D.
  * stress3d   - 3D3V periodic plasma whose per-patch particle counts are drawn
                 log-normal, mirroring the very uneven super-particle counts per
                 process of the 3D run of Sec. 3 (Fig. 2 caption: from 2 570 to
                 6 070 158 per process against 155 520 initially).
Every function returns a plain dict: "params" (grid, time step, boundary and
injection parameters), "particles" (x, y, z, ux, uy, uz, w as float64 and id as
int32, positions physical) and "E", "B" (three float64 arrays each, shape
[ny][nx] or [nz][ny][nx]; B is given at t = +dt/2).
"""
from __future__ import annotations

import math

import numpy as np


def cfl_dt(d, cfl: float = 0.95) -> float:
    """Time step at a fraction of the Yee Courant limit 1/sqrt(sum 1/d^2)."""
    return cfl / math.sqrt(sum(1.0 / (x * x) for x in d))


def _lattice_2d(i0, i1, ny, dx, dy, ppc):
    """Positions of a ppc[0] x ppc[1] lattice in cell columns [i0, i1) x all rows,
    at offsets (a + 1/2)/ppc; ordered row (y) major, then x lattice, as ids."""
    px, py = ppc
    ii = np.arange(i0, i1, dtype=np.float64)
    jj = np.arange(ny, dtype=np.float64)
    ax = (np.arange(px) + 0.5) / px
    by = (np.arange(py) + 0.5) / py
    shape = (jj.size, py, ii.size, px)  # order: j, b, i, a
    x = np.broadcast_to((ii[:, None] + ax[None, :]) * dx, shape)
    y = np.broadcast_to(((jj[:, None] + by[None, :]) * dy)[:, :, None, None], shape)
    return x.ravel(), y.ravel()


def thermal2d(nx: int = 128, ny: int = 128, d: float = 0.1, ppc_side: int = 4,
              uth: float = 0.044, seed: int = 1511, cfl: float = 0.95,
              patch=(32, 32)) -> dict:
    dx = dy = float(d)
    dt = cfl_dt((dx, dy), cfl)
    x, y = _lattice_2d(0, nx, ny, dx, dy, (ppc_side, ppc_side))
    n = x.size
    rng = np.random.default_rng(seed)
    u = rng.normal(0.0, uth, size=(3, n))
    ppc = ppc_side * ppc_side
    w = np.full(n, dx * dy / ppc)
    params = dict(dims=2, n=(nx, ny, 1), d=(dx, dy, 1.0), dt=dt, window=False,
                  q=-1.0, m=1.0, n0=0.0, ramp_x0=0.0, ramp_len=1.0,
                  inject_ppc=(1, 1, 1), patch=tuple(patch), seed=seed,
                  name=f"thermal2d-{nx}x{ny}-ppc{ppc}")
    parts = dict(x=x, y=y, z=np.zeros(n), ux=u[0].copy(), uy=u[1].copy(),
                 uz=u[2].copy(), w=w, id=np.arange(n, dtype=np.int32))
    zeros = [np.zeros((ny, nx)) for _ in range(3)]
    return dict(params=params, particles=parts, E=zeros,
                B=[np.zeros((ny, nx)) for _ in range(3)])


def laser_profile(x, y, a0, w0, tau, xc, yc):
    """Linearly polarised Gaussian pulse, planar phase at focus, k0 = omega0 = 1:
    a0 exp(-(y-yc)^2/w0^2) exp(-2 ln2 (x-xc)^2/tau^2) cos(x - xc); tau is the FWHM
    of the intensity and w0 the 1/e radius of the field."""
    return (a0 * np.exp(-((y - yc) ** 2) / w0 ** 2)
            * np.exp(-2.0 * math.log(2.0) * (x - xc) ** 2 / tau ** 2) * np.cos(x - xc))


def lwfa2d(nx: int = 2048, ny: int = 512, dx: float = 0.125, dy: float = 0.5,
           ppc=(2, 2), n0: float = 0.01, ramp_cells: int = 64, a0: float = 4.0,
           w0: float = 30.0, tau: float = 25.0, laser_back: float = 64.0,
           ramp_x0: float | None = None, seed: int = 1512, cfl: float = 0.95,
           patch=(32, 32)) -> dict:
    """Laser centre x_c = L_x - laser_back; the ramp starts at x_c unless ramp_x0 is
    given (a ramp_x0 far to the left fills the whole window with plasma)."""
    dt = cfl_dt((dx, dy), cfl)
    Lx, Ly = nx * dx, ny * dy
    xc, yc = Lx - laser_back, Ly / 2.0
    if ramp_x0 is None:
        ramp_x0 = xc
    ramp_len = ramp_cells * dx
    x, y = _lattice_2d(0, nx, ny, dx, dy, ppc)
    dens = n0 * np.clip((x - ramp_x0) / ramp_len, 0.0, 1.0)
    keep = dens > 0.0
    x, y, dens = x[keep], y[keep], dens[keep]
    n = x.size
    w = dens * dx * dy / (ppc[0] * ppc[1])
    # Ey on (i, j+1/2) at t = 0; Bz on (i+1/2, j+1/2) at t = +dt/2 (wave moving +x)
    ii = np.arange(nx, dtype=np.float64)[None, :]
    jj = np.arange(ny, dtype=np.float64)[:, None]
    Ey = laser_profile(ii * dx, (jj + 0.5) * dy, a0, w0, tau, xc, yc)
    Bz = laser_profile((ii + 0.5) * dx - 0.5 * dt, (jj + 0.5) * dy, a0, w0, tau, xc, yc)
    E = [np.zeros((ny, nx)), np.ascontiguousarray(Ey), np.zeros((ny, nx))]
    B = [np.zeros((ny, nx)), np.zeros((ny, nx)), np.ascontiguousarray(Bz)]
    params = dict(dims=2, n=(nx, ny, 1), d=(dx, dy, 1.0), dt=dt, window=True,
                  q=-1.0, m=1.0, n0=n0, ramp_x0=float(ramp_x0), ramp_len=ramp_len,
                  inject_ppc=(ppc[0], ppc[1], 1), patch=tuple(patch), seed=seed,
                  a0=a0, w0=w0, tau=tau, xc=xc,
                  name=f"lwfa2d-{nx}x{ny}-ppc{ppc[0] * ppc[1]}")
    parts = dict(x=x, y=y, z=np.zeros(n), ux=np.zeros(n), uy=np.zeros(n),
                 uz=np.zeros(n), w=w, id=np.arange(n, dtype=np.int32))
    return dict(params=params, particles=parts, E=E, B=B)


def _lattice_3d(nx, ny, nz, d, ppc):
    """Positions of a ppc lattice in every cell of an nx x ny x nz grid at offsets
    (a + 1/2)/ppc; ordered (k, j, c, b, i, a) as ids."""
    px, py, pz = ppc
    offs = [(np.arange(p) + 0.5) / p for p in ppc]
    k, j, c, b, i, a = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(pz), np.arange(py),
                                   np.arange(nx), np.arange(px), indexing="ij")
    x = (i + offs[0][a]) * d[0]
    y = (j + offs[1][b]) * d[1]
    z = (k + offs[2][c]) * d[2]
    return x.ravel(), y.ravel(), z.ravel()


def laser_profile3d(x, y, z, a0, w0, tau, xc, yc, zc):
    """The pulse of laser_profile with a round transverse Gaussian in (y, z)."""
    r2 = (y - yc) ** 2 + (z - zc) ** 2
    return (a0 * np.exp(-r2 / w0 ** 2) * np.exp(-2.0 * math.log(2.0) * (x - xc) ** 2 / tau ** 2)
            * np.cos(x - xc))


def lwfa3d(nx: int = 512, ny: int = 128, nz: int = 128, dx: float = 0.125,
           dy: float = 0.5, ppc=(1, 1, 1), n0: float = 0.01, ramp_cells: int = 32,
           a0: float = 4.0, w0: float = 15.0, tau: float = 10.0, laser_back: float = 24.0,
           ramp_x0: float | None = None, seed: int = 1514, cfl: float = 0.95,
           patch=(16, 8, 8)) -> dict:
    """3D LWFA in a moving window (the 3D counterpart of lwfa2d): cold electrons on a
    ppc lattice with the density ramp, a round Gaussian pulse polarised along y
    (E_y at t = 0 on (i, j+1/2, k), B_z at t = +dt/2 on (i+1/2, j+1/2, k))."""
    dz = dy
    d = (dx, dy, dz)
    dt = cfl_dt(d, cfl)
    Lx, Ly, Lz = nx * dx, ny * dy, nz * dz
    xc, yc, zc = Lx - laser_back, Ly / 2.0, Lz / 2.0
    if ramp_x0 is None:
        ramp_x0 = xc
    ramp_len = ramp_cells * dx
    x, y, z = _lattice_3d(nx, ny, nz, d, ppc)
    dens = n0 * np.clip((x - ramp_x0) / ramp_len, 0.0, 1.0)
    keep = dens > 0.0
    x, y, z, dens = x[keep], y[keep], z[keep], dens[keep]
    n = x.size
    w = dens * dx * dy * dz / (ppc[0] * ppc[1] * ppc[2])
    kk = np.arange(nz, dtype=np.float64)[:, None, None]
    jj = np.arange(ny, dtype=np.float64)[None, :, None]
    ii = np.arange(nx, dtype=np.float64)[None, None, :]
    Ey = laser_profile3d(ii * dx, (jj + 0.5) * dy, kk * dz, a0, w0, tau, xc, yc, zc)
    Bz = laser_profile3d((ii + 0.5) * dx - 0.5 * dt, (jj + 0.5) * dy, kk * dz, a0, w0, tau,
                         xc, yc, zc)
    shp = (nz, ny, nx)
    E = [np.zeros(shp), np.ascontiguousarray(np.broadcast_to(Ey, shp)), np.zeros(shp)]
    B = [np.zeros(shp), np.zeros(shp), np.ascontiguousarray(np.broadcast_to(Bz, shp))]
    params = dict(dims=3, n=(nx, ny, nz), d=d, dt=dt, window=True, q=-1.0, m=1.0, n0=n0,
                  ramp_x0=float(ramp_x0), ramp_len=ramp_len, inject_ppc=tuple(ppc),
                  patch=tuple(patch), seed=seed, a0=a0, w0=w0, tau=tau, xc=xc,
                  name=f"lwfa3d-{nx}x{ny}x{nz}-ppc{ppc[0] * ppc[1] * ppc[2]}")
    parts = dict(x=x, y=y, z=z, ux=np.zeros(n), uy=np.zeros(n), uz=np.zeros(n), w=w,
                 id=np.arange(n, dtype=np.int32))
    return dict(params=params, particles=parts, E=E, B=B)


def lognormal_counts(n_patch: int, total: int, sigma: float, rng) -> np.ndarray:
    """Per-patch counts ~ LogNormal(0, sigma) scaled to `total` by largest remainder."""
    L = rng.lognormal(0.0, sigma, size=n_patch)
    share = L / L.sum() * total
    base = np.floor(share).astype(np.int64)
    rem = total - int(base.sum())
    order = np.argsort(-(share - base), kind="stable")
    base[order[:rem]] += 1
    return base


def stress3d(n=(256, 128, 128), d: float = 0.1, patch=(16, 16, 16),
             total: int = 64 * 2 ** 20, sigma: float = 1.5, uth: float = 0.05,
             seed: int = 1513, cfl: float = 0.95) -> dict:
    nx, ny, nz = n
    dx = dy = dz = float(d)
    dt = cfl_dt((dx, dy, dz), cfl)
    px, py, pz = patch
    npx, npy, npz = nx // px, ny // py, nz // pz
    rng = np.random.default_rng(seed)
    counts = lognormal_counts(npx * npy * npz, total, sigma, rng)
    # patch index order: x fastest
    pidx = np.repeat(np.arange(counts.size), counts)
    ox = (pidx % npx) * px
    oy = ((pidx // npx) % npy) * py
    oz = (pidx // (npx * npy)) * pz
    N = int(counts.sum())
    x = (ox + rng.random(N) * px) * dx
    y = (oy + rng.random(N) * py) * dy
    z = (oz + rng.random(N) * pz) * dz
    u = rng.normal(0.0, uth, size=(3, N))
    w = np.full(N, nx * ny * nz * dx * dy * dz / N)
    params = dict(dims=3, n=(nx, ny, nz), d=(dx, dy, dz), dt=dt, window=False,
                  q=-1.0, m=1.0, n0=0.0, ramp_x0=0.0, ramp_len=1.0,
                  inject_ppc=(1, 1, 1), patch=tuple(patch), seed=seed,
                  max_over_mean=float(counts.max() / counts.mean()),
                  name=f"stress3d-{nx}x{ny}x{nz}")
    parts = dict(x=x, y=y, z=z, ux=u[0].copy(), uy=u[1].copy(), uz=u[2].copy(), w=w,
                 id=np.arange(N, dtype=np.int32))
    shp = (nz, ny, nx)
    return dict(params=params, particles=parts,
                E=[np.zeros(shp) for _ in range(3)], B=[np.zeros(shp) for _ in range(3)])
