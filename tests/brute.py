"""Brute-force recomputation of the CPM state functions, for tests.

Written straight from the definitions (Methods, Eq. 1 and Eq. 3) with numpy
whole-lattice operations, with no incremental bookkeeping: the full
Hamiltonian, per-cell volumes and per-cell interface counts.  Used to pin the
oracle's incremental energy changes and tallies.
"""
import itertools

import numpy as np


def offsets(dim):
    rng = [-1, 0, 1]
    if dim == 2:
        return [(0, dy, dx) for dy in rng for dx in rng if (dy, dx) != (0, 0)]
    return [(dz, dy, dx) for dz, dy, dx in itertools.product(rng, rng, rng) if (dz, dy, dx) != (0, 0, 0)]


def types_of(w, lat):
    t = np.where(lat < 0, w.obstacle_type, w.cell_type[np.maximum(lat, 0)])
    return t.astype(np.int64)


def volumes(w, lat):
    return np.bincount(lat[lat > 0].ravel(), minlength=w.n_cells + 1).astype(np.int64)


def interfaces(w, lat):
    A = np.zeros(w.n_cells + 1, dtype=np.int64)
    for o in offsets(w.dim):
        nb = np.roll(lat, shift=tuple(-x for x in o), axis=(0, 1, 2))
        m = (lat > 0) & (nb != lat)
        A += np.bincount(lat[m].ravel(), minlength=w.n_cells + 1)
    return A


def hamiltonian(w, lat):
    """Eq. 1 (each unordered neighbour pair once) plus the perimeter term."""
    tp = types_of(w, lat)
    adh = 0
    for o in offsets(w.dim):
        nb = np.roll(lat, shift=tuple(-x for x in o), axis=(0, 1, 2))
        tn = np.roll(tp, shift=tuple(-x for x in o), axis=(0, 1, 2))
        diff = nb != lat
        adh += int(w.J[tp[diff], tn[diff]].astype(np.int64).sum())
    assert adh % 2 == 0
    adh //= 2
    V = volumes(w, lat)
    A = interfaces(w, lat)
    ids = np.arange(1, w.n_cells + 1)
    ct = w.cell_type[ids].astype(np.int64)
    vol = int((w.lambda_v[ct].astype(np.int64) * (V[ids] - w.v_target[ct]) ** 2).sum())
    per = int((w.lambda_p[ct].astype(np.int64) * (A[ids] - w.a_target[ct]) ** 2).sum())
    return adh + vol + per


def hamiltonian_batch(w, lats):
    """Same as ``hamiltonian`` for a batch of lattices [B, nz, ny, nx] with a
    handful of cells (loops over cell ids, vectorised over the batch)."""
    lats = np.asarray(lats)
    B = lats.shape[0]
    tp = np.where(lats < 0, w.obstacle_type, w.cell_type[np.maximum(lats, 0)]).astype(np.int64)
    adh = np.zeros(B, dtype=np.int64)
    nbs = []
    for o in offsets(w.dim):
        sh = tuple(-x for x in o)
        nb = np.roll(lats, shift=sh, axis=(1, 2, 3))
        tn = np.roll(tp, shift=sh, axis=(1, 2, 3))
        diff = nb != lats
        adh += np.where(diff, w.J[tp, tn], 0).reshape(B, -1).sum(1)
        nbs.append(nb)
    assert np.all(adh % 2 == 0)
    H = adh // 2
    for cid in range(1, w.n_cells + 1):
        ct = int(w.cell_type[cid])
        mine = lats == cid
        V = mine.reshape(B, -1).sum(1)
        A = sum((mine & (nb != cid)).reshape(B, -1).sum(1) for nb in nbs)
        H = H + int(w.lambda_v[ct]) * (V - int(w.v_target[ct])) ** 2
        H = H + int(w.lambda_p[ct]) * (A - int(w.a_target[ct])) ** 2
    return H
