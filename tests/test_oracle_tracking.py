"""Pins of the oracle's composite variable tracking (Methods, "Composite
variable tracking", Eq. 10 and Eq. 11) to the lattice it describes.

The replay keeps, per cell, the integer sums S of its sites' coordinates
beside its size V, so that the centroid is S / V.  Under periodic
boundaries each site counts at its periodic image nearest the cell's
centroid.  Checked here against things other than the tracking code:

* a hand-made cell straddling the lattice corner (closed form);
* after replays with cells drifting across the periodic boundary: every
  cell's sites, each placed at its image nearest S / V by a brute-force
  numpy recomputation, sum to S exactly, and V is the site count;
* at MCS ends the centroid lies in [0, n) and equals the snapshot centroid
  of the lattice (Eq. 10, computed from the lattice alone) modulo n;
* tracking changes nothing in the dynamics (the lattice is that of a replay
  without it).
"""
import numpy as np
import pytest

import cpm_workloads as cw
import oracle


def coords(w, lat):
    """(ids, x, y, z) of every site of a lattice in the oracle's x-fastest order."""
    z, y, x = np.meshgrid(np.arange(w.nz), np.arange(w.ny), np.arange(w.nx), indexing="ij")
    return lat.reshape(-1), x.reshape(-1), y.reshape(-1), z.reshape(-1)


def brute_sums(w, lat, S):
    """Per cell: the sum of its sites' coordinates, each at the periodic image
    nearest S / V, and the site count; integer arithmetic throughout."""
    ids, x, y, z = coords(w, lat)
    ext = (w.nx, w.ny, w.nz)
    out = np.zeros_like(S)
    cnt = np.bincount(ids[ids > 0], minlength=w.n_cells + 1)
    for c in range(1, w.n_cells + 1):
        m = ids == c
        V = int(cnt[c])
        if V == 0:
            continue
        for d, q in enumerate((x, y, z)[:w.dim]):
            qc = q[m].astype(np.int64)
            k = np.floor_divide(2 * (S[c, d] - qc * V) + ext[d] * V, 2 * ext[d] * V)
            out[c, d] = int(np.sum(qc + ext[d] * k))
    return out, cnt


def straddles(w, lat):
    """Whether some cell has sites in both the first and the last plane of an axis."""
    ids, x, y, z = coords(w, lat)
    for d, q in enumerate((x, y, z)[:w.dim]):
        n = (w.nx, w.ny, w.nz)[d]
        lo = set(ids[(q == 0) & (ids > 0)].tolist())
        hi = set(ids[(q == n - 1) & (ids > 0)].tolist())
        if lo & hi:
            return True
    return False


def test_hand_cells_across_the_corner():
    w = cw.random_small(1, dim=2, n=16, n_cells=2, edge=1)
    lat = np.zeros((1, 16, 16), dtype=np.int32)
    for (x, y) in [(15, 15), (0, 15), (15, 0), (0, 0)]:
        lat[0, y, x] = 1                       # a 2x2 cell around the corner
    for x in (15, 0, 1):
        lat[0, 5, x] = 2                       # a 3x1 cell across x = 0
    w = w.replace(lattice=lat, act=None)
    st = oracle.State(w, track=True)
    # cell 1: centroid (-0.5, -0.5) moved into bounds: (15.5, 15.5), S = V * centroid
    assert st.csum[1, :2].tolist() == [62, 62]
    # cell 2: images -1, 0, 1 along x: centroid (0, 5)
    assert st.csum[2, :2].tolist() == [0, 15]
    assert st.V[1] == 4 and st.V[2] == 3
    assert np.all(st.csum[:, 2] == 0)


def drifting(dim, seed, act):
    """Small cells pushed along a constant chemotactic field, so that they
    cross the periodic boundary within a few tens of MCS."""
    if dim == 2:
        w = cw.random_small(seed, dim=2, n=24, n_cells=10, edge=3, act=act, T=20.0)
        f = cw.uniform_field((1, 24, 24), 2, (1.0, 0.35))
    else:
        w = cw.random_small(seed, dim=3, n=12, n_cells=6, edge=3, act=act, T=20.0)
        f = cw.uniform_field((12, 12, 12), 3, (1.0, 0.4, 0.2))
    return cw.with_motility(w, chem=f, lambda_chem=400)


def obstructed_3d():
    """3D cells among frozen obstacle sites on 8^3 areas (a second block size and schedule)."""
    w = cw.random_small(12, dim=3, n=16, n_cells=10, edge=3, act=True, obstacles=0.04, a=8, c=2, P=16)
    return cw.with_motility(w, chem=cw.uniform_field((16, 16, 16), 3, (0.2, 1.0, 0.5)), lambda_chem=300)


@pytest.mark.parametrize("dim,seed,act", [(2, 3, False), (2, 4, True), (3, 5, True), (3, 0, True)])
def test_tracked_sums_follow_the_lattice(dim, seed, act):
    w = drifting(dim, seed, act) if seed else obstructed_3d()
    st = oracle.State(w, track=True)
    plain = oracle.State(w)
    per = st.subpasses_per_mcs()
    ext = np.array([w.nx, w.ny, w.nz], dtype=np.float64)
    crossed = straddles(w, st.lattice)
    # uneven steps, so that checks fall in the middle of MCS as well as at their ends
    steps = [3, per - 3, 1, per - 1] + [per] * 26
    for n_sub in steps:
        st.replay_subpasses(n_sub)
        plain.replay_subpasses(n_sub)
        assert np.array_equal(st.lattice, plain.lattice), "tracking changed the dynamics"
        S_b, cnt = brute_sums(w, st.lattice, st.csum)
        live = cnt > 0
        live[0] = False
        assert np.array_equal(st.V[live], cnt[live])
        assert np.array_equal(st.csum[live], S_b[live])
        assert np.all(st.csum[cnt == 0] == 0), "a cell without sites kept non-zero sums"
        crossed = crossed or straddles(w, st.lattice)
        if st.sp == 0:
            X = st.csum[live, :dim] / st.V[live, None]
            assert np.all(X >= 0) and np.all(X < ext[:dim])
            Xs = st.centroids()[live, :dim]
            diff = np.mod(X - Xs + ext[:dim] / 2, ext[:dim]) - ext[:dim] / 2
            assert np.max(np.abs(diff)) < 1e-9
    assert crossed, "no cell met the periodic boundary: the case this test is for was not exercised"


def test_planted_raw_coordinates_fail_the_pin():
    """Summing raw coordinates (no periodic image) breaks the brute-force
    check for a cell across the boundary, so the pin can fail."""
    w = cw.random_small(1, dim=2, n=16, n_cells=2, edge=1)
    lat = np.zeros((1, 16, 16), dtype=np.int32)
    for x in (15, 0, 1):
        lat[0, 5, x] = 1
    w = w.replace(lattice=lat, act=None)
    raw = np.zeros((w.n_cells + 1, 3), dtype=np.int64)
    raw[1, :2] = [15 + 0 + 1, 15]
    S_b, _ = brute_sums(w, lat, raw)
    assert not np.array_equal(S_b[1], raw[1])
