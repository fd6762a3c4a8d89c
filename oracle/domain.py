"""Ownership and ghost sets of the spatial decomposition -- TEST INFRASTRUCTURE ONLY.

Only the test-suite may import this module.  It writes out, in plain numpy
FP64, what the library's domain kernels must compute bit for bit for a 3-D
multi-section geometry (Sec. II of the paper: rectangular domains, one per
process; the short-range force vanishes beyond r_cut, so a domain needs the
particles within r_cut of its box as well as its own):

  geometry   nx slabs cut along x at xc[0..nx]; slab i cut along y at
             yc[i][0..ny]; column (i, j) cut along z at zc[i][j][0..nz];
             domain d = (i ny + j) nz + k is the half-open box
             [xc[i], xc[i+1]) x [yc[i][j], yc[i][j+1]) x [zc[i][j][k], zc[i][j][k+1])
  wrap       x - floor(x), with 1.0 -> 0.0 (as the tree wraps positions)
  owner      along each axis the largest cut <= the coordinate (slab, then
             column within the slab, then cell within the column)
  ghost      particle p goes to domain d (d not its own) when the squared
             periodic distance from p to d's box is below r_cut^2; per axis
             the distance is 0 inside [lo, hi), else the shorter way round:
             min(lo - p, (p + 1) - hi) for p < lo, min(p - hi, (lo + 1) - p)
             for p >= hi; squared distance (gx gx + gy gy) + gz gz, every
             operation rounded separately
  order      per destination domain (domain 0 first) the particle indices in
             ascending order
"""
from __future__ import annotations

import numpy as np


def wrap(pos: np.ndarray) -> np.ndarray:
    w = pos - np.floor(pos)
    w[w >= 1.0] = 0.0
    return w


def boxes(xc, yc, zc):
    """lo, hi [ndom, 3] of every domain, in domain order."""
    xc, yc, zc = np.asarray(xc), np.asarray(yc), np.asarray(zc)
    nx, ny, nz = xc.size - 1, yc.shape[1] - 1, zc.shape[2] - 1
    lo = np.zeros((nx * ny * nz, 3))
    hi = np.zeros((nx * ny * nz, 3))
    for i in range(nx):
        for j in range(ny):
            for k in range(nz):
                d = (i * ny + j) * nz + k
                lo[d] = (xc[i], yc[i, j], zc[i, j, k])
                hi[d] = (xc[i + 1], yc[i, j + 1], zc[i, j, k + 1])
    return lo, hi


def owner(pos, xc, yc, zc) -> np.ndarray:
    """The domain holding each particle (after wrapping)."""
    xc, yc, zc = np.asarray(xc), np.asarray(yc), np.asarray(zc)
    nx, ny, nz = xc.size - 1, yc.shape[1] - 1, zc.shape[2] - 1
    w = wrap(np.asarray(pos, dtype=np.float64))
    i = np.minimum(np.searchsorted(xc, w[:, 0], side="right") - 1, nx - 1)
    j = np.zeros_like(i)
    k = np.zeros_like(i)
    for a in range(nx):
        sa = i == a
        j[sa] = np.minimum(np.searchsorted(yc[a], w[sa, 1], side="right") - 1, ny - 1)
        for b in range(ny):
            sb = sa & (j == b)
            k[sb] = np.minimum(np.searchsorted(zc[a, b], w[sb, 2], side="right") - 1, nz - 1)
    return ((i * ny + j) * nz + k).astype(np.int64)


def axis_gap(p: np.ndarray, lo: float, hi: float) -> np.ndarray:
    below = np.minimum(lo - p, (p + 1.0) - hi)
    above = np.minimum(p - hi, (lo + 1.0) - p)
    return np.where(p < lo, below, np.where(p >= hi, above, 0.0))


def near(pos, lo, hi, r_cut) -> np.ndarray:
    """Particles whose squared periodic distance to the box [lo, hi) is below r_cut^2."""
    w = wrap(np.asarray(pos, dtype=np.float64))
    gx = axis_gap(w[:, 0], lo[0], hi[0])
    gy = axis_gap(w[:, 1], lo[1], hi[1])
    gz = axis_gap(w[:, 2], lo[2], hi[2])
    return (gx * gx + gy * gy) + gz * gz < r_cut * r_cut


def select(pos, xc, yc, zc, mode: str, self_domain: int = -1, r_cut: float = 0.0):
    """Indices grouped by destination domain (ascending within each) and the
    count per destination.  mode "owner": every particle to its owner;
    mode "ghosts": every particle to every domain other than self_domain whose
    box is within r_cut of it."""
    lo, hi = boxes(xc, yc, zc)
    nd = lo.shape[0]
    if mode == "owner":
        own = owner(pos, xc, yc, zc)
        lists = [np.nonzero(own == d)[0] for d in range(nd)]
    elif mode == "ghosts":
        lists = [np.zeros(0, dtype=np.int64) if d == self_domain else np.nonzero(near(pos, lo[d], hi[d], r_cut))[0]
                 for d in range(nd)]
    else:
        raise ValueError(mode)
    counts = np.array([l.size for l in lists], dtype=np.int64)
    idx = np.concatenate(lists) if lists else np.zeros(0, dtype=np.int64)
    return idx.astype(np.int64), counts
