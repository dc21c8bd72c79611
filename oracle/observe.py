"""Lattice observations behind the emulator's summary statistics: test
infrastructure only (imported by ``tests/`` and never by the library).

* Cell centroids on the periodic lattice, following the paper's composite
  variable tracking (Methods, "Composite variable tracking", Eq. 10): a
  centroid is the mean of the cell's site coordinates, taken on a periodic
  image that keeps the cell in one piece.  The image is fixed here by an
  anchor, the cell's first site in raster order (z, y, x): every coordinate
  is replaced by the anchor's plus the minimal-image offset
  ((p - anchor + L/2) mod L) - L/2, so the per-cell sums are integers.
* Interface pairs between a cell and the medium (id 0), counted once per
  unordered neighbour pair over the model's neighbourhood (Moore in 2D, 26
  neighbours in 3D); together with the per-cell interface tallies they give
  the number of cell-cell pairs.

Plain numpy loops over cells; small lattices only.
"""
from __future__ import annotations

import itertools

import numpy as np


def centroid_sums(lat, n_cells):
    """Per cell id 1..n_cells: (anchor linear index, count, offset sums per
    axis in (x, y, z) order), all integers; anchor -1 and zeros for an empty
    cell.  ``lat`` has shape (nz, ny, nx)."""
    lat = np.asarray(lat)
    nz, ny, nx = lat.shape
    L = np.array([nx, ny, nz], dtype=np.int64)
    anchor = np.full(n_cells + 1, -1, dtype=np.int64)
    count = np.zeros(n_cells + 1, dtype=np.int64)
    sums = np.zeros((n_cells + 1, 3), dtype=np.int64)
    flat = lat.ravel()
    for c in range(1, n_cells + 1):
        idx = np.nonzero(flat == c)[0]
        if idx.size == 0:
            continue
        a = int(idx[0])
        anchor[c] = a
        count[c] = idx.size
        z, rem = np.divmod(idx, ny * nx)
        y, x = np.divmod(rem, nx)
        az, ar = divmod(a, ny * nx)
        ay, ax = divmod(ar, nx)
        for d, (p, q) in enumerate(((x, ax), (y, ay), (z, az))):
            off = np.mod(p - q + L[d] // 2, L[d]) - L[d] // 2
            sums[c, d] = int(off.sum())
    return anchor, count, sums


def centroids(lat, n_cells):
    """Float centroids (x, y, z) per cell from ``centroid_sums``, wrapped
    into the lattice; NaN for empty cells."""
    lat = np.asarray(lat)
    nz, ny, nx = lat.shape
    anchor, count, sums = centroid_sums(lat, n_cells)
    out = np.full((n_cells + 1, 3), np.nan)
    for c in range(1, n_cells + 1):
        if count[c] == 0:
            continue
        az, ar = divmod(int(anchor[c]), ny * nx)
        ay, ax = divmod(ar, nx)
        out[c] = np.mod(np.array([ax, ay, az], float) + sums[c] / count[c], [nx, ny, nz])
    return out


def cell_medium_pairs(lat, dim):
    """Unordered neighbour pairs (cell > 0, medium 0) on the periodic
    lattice, over the Moore (2D) or 26 (3D) neighbourhood."""
    lat = np.asarray(lat)
    if dim == 2:
        g = lat[0]
        offs = [(dy, dx) for dy, dx in itertools.product((-1, 0, 1), repeat=2) if (dy, dx) != (0, 0)]
        n = 0
        for dy, dx in offs:
            nb = np.roll(g, (-dy, -dx), axis=(0, 1))
            n += int(((g > 0) & (nb == 0)).sum())
        return n
    offs = [o for o in itertools.product((-1, 0, 1), repeat=3) if o != (0, 0, 0)]
    n = 0
    for o in offs:
        nb = np.roll(lat, tuple(-x for x in o), axis=(0, 1, 2))
        n += int(((lat > 0) & (nb == 0)).sum())
    return n
