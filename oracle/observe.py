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

Plain numpy loops over cells; small lattices only.  ``summary_statistics``
reduces stacked observations of many runs to the emulator's sixteen targets.
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


def cell_rows(lat, n_cells, dim):
    """Per cell id 0..n_cells a row of 12 integers: anchor (-1 if empty),
    volume, offset sums (x, y, z), interface count (neighbours with another
    id, Eq. 3), and offset product sums xx, yy, zz, xy, xz, yz; row 0 (the
    medium) is [-1, 0, ...]."""
    lat = np.asarray(lat)
    nz, ny, nx = lat.shape
    L = np.array([nx, ny, nz], dtype=np.int64)
    rows = np.zeros((n_cells + 1, 12), dtype=np.int64)
    rows[:, 0] = -1
    if dim == 2:
        offs = [(0, dy, dx) for dy, dx in itertools.product((-1, 0, 1), repeat=2) if (dy, dx) != (0, 0)]
    else:
        offs = [o for o in itertools.product((-1, 0, 1), repeat=3) if o != (0, 0, 0)]
    differ = np.zeros(lat.shape, dtype=np.int64)
    for o in offs:
        differ += np.roll(lat, tuple(-x for x in o), axis=(0, 1, 2)) != lat
    flat = lat.ravel()
    dflat = differ.ravel()
    for c in range(1, n_cells + 1):
        idx = np.nonzero(flat == c)[0]
        if idx.size == 0:
            continue
        a = int(idx[0])
        z, rem = np.divmod(idx, ny * nx)
        y, x = np.divmod(rem, nx)
        az, ar = divmod(a, ny * nx)
        ay, ax = divmod(ar, nx)
        off = [np.mod(p - q + L[d] // 2, L[d]) - L[d] // 2 for d, (p, q) in enumerate(((x, ax), (y, ay), (z, az)))]
        ox, oy, oz = off
        rows[c] = [a, idx.size, ox.sum(), oy.sum(), oz.sum(), dflat[idx].sum(),
                   (ox * ox).sum(), (oy * oy).sum(), (oz * oz).sum(), (ox * oy).sum(), (ox * oz).sum(),
                   (oy * oz).sum()]
    return rows


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


# --------------------------------------------------------------------------
# summary statistics of runs (the emulator's targets)
# --------------------------------------------------------------------------

SUMMARY_STATS = ["vol_mean", "vol_sd", "perim_mean", "perim_sd", "msd10", "msd50", "msd200", "speed_mean",
                 "speed_sd", "dac50", "persistence", "arrest", "acceptance", "contact_cc", "straightness",
                 "elongation"]
ARREST_SPEED = 0.05  # sites / MCS over a 50-MCS sub-track


def _masked_mean(x, m, axis):
    s = np.where(m, x, 0.0).sum(axis=axis)
    c = m.sum(axis=axis)
    with np.errstate(invalid="ignore", divide="ignore"):
        return s / c


def summary_statistics(cells, member, n_cells, shape, v_target, a_target, every, n_sites):
    """The sixteen summary statistics (SUMMARY_STATS order) of runs with
    equal geometry, written out with numpy over whole arrays.

    cells:  int64 [S+1, n_runs, n_cells+1, 12], cpm_batch_observe rows per
            snapshot (snapshots ``every`` MCS apart);
    member: int64 [S+1, n_runs, 2] (cell-medium pairs, accepted copies);
    shape:  (nx, ny) of the 2D lattice.  Returns float64 [n_runs, 16]; NaN
    where a statistic is undefined (no surviving cell, too short a window).
    """
    cells = np.asarray(cells)[:, :, 1:, :].astype(np.float64)
    member = np.asarray(member).astype(np.float64)
    S1, n = cells.shape[0], cells.shape[1]
    nx, ny = shape
    L = np.array([nx, ny], dtype=np.float64)
    anchor, V, A = cells[..., 0], cells[..., 1], cells[..., 5]
    alive = V > 0
    out = np.full((n, len(SUMMARY_STATS)), np.nan)
    # statistics scaled by a target of 0 (no such constraint) stay NaN (undefined)
    if v_target != 0:
        out[:, 0] = _masked_mean(V, alive, (0, 2)) / v_target
    if a_target != 0:
        out[:, 2] = _masked_mean(A, alive, (0, 2)) / a_target
    with np.errstate(invalid="ignore", divide="ignore"):
        vm = _masked_mean(V, alive, 2)
        am = _masked_mean(A, alive, 2)
        vv = _masked_mean((V - vm[..., None]) ** 2, alive, 2)
        av = _masked_mean((A - am[..., None]) ** 2, alive, 2)
    if v_target != 0:
        out[:, 1] = np.sqrt(np.nanmean(vv, axis=0)) / v_target
    if a_target != 0:
        out[:, 3] = np.sqrt(np.nanmean(av, axis=0)) / a_target
    # centroids: anchor + offset mean, unwrapped across snapshots
    Vs = np.where(alive, V, 1.0)
    ax = np.mod(anchor, nx)
    ay = np.floor_divide(anchor, nx)
    c = np.stack([ax + cells[..., 2] / Vs, ay + cells[..., 3] / Vs], axis=-1)  # [S1, n, C, 2]
    d = np.diff(c, axis=0)
    d -= L * np.round(d / L)
    traj = np.concatenate([np.zeros_like(c[:1]), np.cumsum(d, axis=0)], axis=0)
    track = alive.all(axis=0)  # cells alive at every snapshot  [n, C]

    def lag_disp(k):
        return traj[k:] - traj[:-k]

    for col, lag in ((4, 10), (5, 50), (6, 200)):
        k = lag // every
        if 0 < k < S1 and lag % every == 0:
            sq = (lag_disp(k) ** 2).sum(-1)
            out[:, col] = _masked_mean(sq, np.broadcast_to(track[None], sq.shape), (0, 2))
    steps = lag_disp(1) if S1 > 1 else None
    if steps is not None:
        sp = np.sqrt((steps ** 2).sum(-1)) / every
        m = np.broadcast_to(track[None], sp.shape)
        out[:, 7] = _masked_mean(sp, m, (0, 2))
        out[:, 8] = np.sqrt(_masked_mean((sp - out[:, 7][None, :, None]) ** 2, m, (0, 2)))
        # step-direction autocorrelation; persistence = every * (1/2 + sum of C_k up to the first C_k <= 0)
        nrm = np.sqrt((steps ** 2).sum(-1))
        u = np.where(nrm[..., None] > 0, steps / np.maximum(nrm, 1e-12)[..., None], 0.0)
        ok = (nrm > 0) & track[None]
        pers = np.full(n, 0.5 * every)
        running = np.ones(n, dtype=bool)
        for k in range(1, min(21, S1 - 1)):
            cos = (u[k:] * u[:-k]).sum(-1)
            Ck = _masked_mean(cos, ok[k:] & ok[:-k], (0, 2))
            Ck = np.nan_to_num(Ck, nan=0.0)
            running &= Ck > 0
            pers += np.where(running, Ck * every, 0.0)
        out[:, 10] = pers
        path = nrm.sum(0)  # [n, C]
        net = np.sqrt((traj[-1] ** 2).sum(-1))
        with np.errstate(invalid="ignore", divide="ignore"):
            st = net / path
        out[:, 14] = _masked_mean(st, track & (path > 0), 1)
    k50 = 50 // every
    if 50 % every == 0 and 2 * k50 < S1:
        d50 = lag_disp(k50)
        n50 = np.sqrt((d50 ** 2).sum(-1))
        a, b = d50[k50:], d50[:-k50]
        na, nb = n50[k50:], n50[:-k50]
        with np.errstate(invalid="ignore", divide="ignore"):
            cos = (a * b).sum(-1) / (na * nb)
        okc = (na > 0) & (nb > 0) & track[None]
        out[:, 9] = _masked_mean(np.nan_to_num(cos), okc, (0, 2))
        slow = (n50 / 50.0) < ARREST_SPEED
        out[:, 11] = _masked_mean(slow.astype(np.float64), np.broadcast_to(track[None], slow.shape), (0, 2))
    out[:, 12] = (member[-1, :, 1] - member[0, :, 1]) / ((S1 - 1) * every * n_sites)
    sumA = np.where(alive, A, 0.0).sum(-1)  # [S1, n]
    cm = member[..., 0]
    cc = (sumA - cm) / 2.0
    tot = cc + cm
    out[:, 13] = _masked_mean(cc / np.where(tot > 0, tot, 1.0), tot > 0, 0)
    # elongation from the second moments about the centroid
    mx, my = cells[..., 2] / Vs, cells[..., 3] / Vs
    cxx = cells[..., 6] / Vs - mx * mx
    cyy = cells[..., 7] / Vs - my * my
    cxy = cells[..., 9] / Vs - mx * my
    tr, det = cxx + cyy, cxx * cyy - cxy * cxy
    disc = np.sqrt(np.maximum(tr * tr / 4 - det, 0.0))
    l1, l2 = tr / 2 + disc, tr / 2 - disc
    with np.errstate(invalid="ignore", divide="ignore"):
        el = np.sqrt(l1 / l2)
    oke = alive & (l2 > 1e-9)
    out[:, 15] = _masked_mean(np.where(oke, el, 0.0), oke, (0, 2))
    return out
