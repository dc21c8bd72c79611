"""Pins of the CPU oracle to things other than itself.

* Philox4x32-10 against its published known-answer vectors.
* The threshold, log and exp tables against the exact functions within the
  error bound of their rounding.
* Integer energy changes against a brute-force recomputation of the full
  Hamiltonian (Methods, Eq. 1 and Eq. 3) before and after the copy.
* Tallies against a recount after runs of both oracles.
* Act geometric means against closed forms (constant Act, a zero, medium).
* The schedule of the parallel replay against the closed form of its update
  statistics (Results, Fig. 3: one attempt per site per MCS on average, a
  binomial count per MCS) and the colour order against uniform permutations.
"""
import math
import os

import numpy as np
import pytest

import cpm_workloads as cw
import oracle
from tests import brute

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_philox_known_answers():
    rows = [l.split() for l in open(os.path.join(GOLDEN, "philox4x32_10_kat.txt"))
            if l.strip() and not l.startswith("#")]
    assert len(rows) == 3
    for r in rows:
        v = [int(x, 16) for x in r]
        assert oracle.philox4x32_10(v[0:4], v[4:6]) == v[6:10]


@pytest.mark.parametrize("T", [20.0, 40.0, 100.0, 7.5])
def test_threshold_table_bounds(T):
    thr = oracle.thr_table(T).astype(np.float64)
    h = np.arange(len(thr), dtype=np.float64)
    exact = np.exp(-h / (16.0 * T)) * 2.0 ** 32
    # floor of the exact value, up to one unit from exp's own rounding
    assert np.all(thr <= np.minimum(exact, 2.0 ** 32 - 1) + 1)
    assert np.all(thr >= exact - 2)
    assert thr[0] == 2 ** 32 - 1
    assert np.all(np.diff(thr) <= 0)
    assert np.all(thr > 0)
    # the table ends where 2^32 exp(-h/16T) drops below 1
    L = len(thr)
    assert abs(L - 16.0 * T * 32.0 * math.log(2.0)) <= 2


def test_log_and_exp_tables():
    ln = oracle.ln_table()
    a = np.arange(1, 129)
    assert np.all(np.abs(ln[1:] - np.log(a) * 65536.0) <= 0.5 + 1e-9)
    assert ln[1] == 0
    ex = oracle.expq_table()
    m = np.arange(len(ex))
    assert np.all(np.abs(ex - np.exp(m / 1024.0) * 65536.0) <= 0.5 + 1e-6)
    assert ex[0] == 65536
    assert len(ex) == (ln[128] >> 6) + 1


def _random_attempts(w, st, rng, n):
    off = oracle.neighbour_offsets(w.dim)
    N = w.n_sites
    out = []
    tries = 0
    while len(out) < n and tries < 100 * n:
        tries += 1
        j = int(rng.integers(N))
        k = int(rng.integers(len(off)))
        z, y, x = np.unravel_index(j, st.lattice.shape)
        dx, dy, dz = off[k]
        i = np.ravel_multi_index(((z + dz) % w.nz, (y + dy) % w.ny, (x + dx) % w.nx), st.lattice.shape)
        si, sj = st.lattice.flat[i], st.lattice.flat[j]
        if si == sj or si < 0 or sj < 0:
            continue
        if sj > 0 and st.V[sj] <= 1:
            continue
        out.append((j, k, int(si)))
    return out


@pytest.mark.parametrize("dim,seed,obst", [(2, 1, 0.0), (2, 2, 0.1), (3, 3, 0.0), (3, 4, 0.08)])
def test_delta_h_equals_full_hamiltonian_difference(dim, seed, obst):
    w = cw.random_small(seed, dim=dim, n=8 if dim == 3 else 12, n_cells=6, edge=3, perimeter=True,
                        obstacles=obst, n_types=2)
    st = oracle.State(w)
    rng = np.random.default_rng(seed)
    st.replay_run(2)  # move away from cubes
    checked = 0
    for j, k, si in _random_attempts(w, st, rng, 60):
        d = st.delta_h(j, k)
        before = brute.hamiltonian(w, st.lattice)
        lat2 = st.lattice.copy()
        lat2.flat[j] = si
        after = brute.hamiltonian(w, lat2)
        assert d["dh_int"] == after - before, (j, k)
        checked += 1
    assert checked >= 30


@pytest.mark.parametrize("mode", ["serial", "replay"])
@pytest.mark.parametrize("dim,act,obst", [(2, False, 0.0), (2, True, 0.05), (3, False, 0.05), (3, True, 0.0)])
def test_tallies_match_recount(mode, dim, act, obst):
    w = cw.random_small(11 + dim, dim=dim, n=8 if dim == 3 else 16, n_cells=8, edge=3,
                        perimeter=True, act=act, obstacles=obst, T=40.0)
    st = oracle.State(w)
    for _ in range(3):
        if mode == "serial":
            st.serial_run(2)
        else:
            st.replay_run(2)
        V = brute.volumes(w, st.lattice)
        A = brute.interfaces(w, st.lattice)
        assert np.array_equal(V, st.V.astype(np.int64))
        assert np.array_equal(A, st.A.astype(np.int64))
        assert np.all(st.lattice[w.lattice < 0] == -1)        # obstacles frozen
        assert np.all((st.lattice >= 0) | (w.lattice < 0))    # nothing new is frozen
        if act:
            mx = w.max_act[w.cell_type[np.maximum(st.lattice, 0)]]
            assert np.all(st.act <= np.where(st.lattice > 0, mx, 0))


def _act_lattice(dim, act_value):
    w = cw.random_small(5, dim=dim, n=8, n_cells=1, edge=5, perimeter=False, act=True, n_types=1)
    w.max_act[1] = 60
    st = oracle.State(w)
    st.act[:] = 0
    st.act[st.lattice > 0] = act_value
    return w, st


@pytest.mark.parametrize("dim", [2, 3])
def test_act_geometric_mean_closed_forms(dim):
    w, st = _act_lattice(dim, 37)
    cell = np.flatnonzero(st.lattice.ravel() > 0)
    med = np.flatnonzero(st.lattice.ravel() == 0)
    off = oracle.neighbour_offsets(dim)
    # a target inside the cell next to the medium: GM(j) over a constant Act is that constant
    found = False
    for j in cell:
        for k in range(len(off)):
            d = st.delta_h(int(j), k)
            z, y, x = np.unravel_index(j, st.lattice.shape)
            dx, dy, dz = off[k]
            i = np.ravel_multi_index(((z + dz) % w.nz, (y + dy) % w.ny, (x + dx) % w.nx), st.lattice.shape)
            if st.lattice.flat[i] == 0:
                assert d["gm_j"] == pytest.approx(37.0, rel=1e-12)
                assert d["gm_i"] == 0.0 and d["gm_i_q"] == 0
                assert abs(d["gm_j_q"] / 65536.0 - 37.0) <= 37.0 * 2e-3
                # medium source: lambda and Max of the target's type
                lam, mx = w.lambda_act[1], w.max_act[1]
                assert d["dh_act_real"] == pytest.approx(lam / mx * 37.0, rel=1e-12)
                assert abs(d["dh_act_q"] - 16 * d["dh_act_real"]) <= 1 + 16 * lam / mx * 37.0 * 2e-3
                found = True
                break
        if found:
            break
    assert found
    # one zero in the same-cell neighbourhood makes the mean zero
    st.act.flat[cell[len(cell) // 2]] = 0
    j = int(cell[len(cell) // 2])
    d = st.delta_h(j, 0)
    assert d["gm_j"] == 0.0 and d["gm_j_q"] == 0
    assert len(med) > 0


@pytest.mark.parametrize("dim", [2, 3])
def test_act_integer_mean_within_rounding_bound(dim):
    """Integer GM (tables) against the real GM, for random Act values."""
    rng = np.random.default_rng(dim)
    for rep in range(4):
        w = cw.random_small(40 + rep, dim=dim, n=8 if dim == 3 else 12, n_cells=5, edge=4,
                            perimeter=True, act=True, n_types=2)
        st = oracle.State(w)
        st.act[st.lattice > 0] = rng.integers(1, 61, size=int((st.lattice > 0).sum()))
        for j, k, si in _random_attempts(w, st, rng, 30):
            d = st.delta_h(j, k)
            for a, b in (("gm_i", "gm_i_q"), ("gm_j", "gm_j_q")):
                assert abs(d[b] / 65536.0 - d[a]) <= d[a] * 1.5e-3 + 1e-12
            tp = 1 if si == 0 else 0
            lam_mx = max(w.lambda_act[1:3] / np.maximum(w.max_act[1:3], 1))
            bound = 1 + 16 * lam_mx * 1.5e-3 * (d["gm_i"] + d["gm_j"])
            assert abs(d["dh_act_q"] - 16 * d["dh_act_real"]) <= bound
            del tp


@pytest.mark.parametrize("dim,a,c,P", [(2, 4, 2, 1), (2, 8, 2, 2), (3, 8, 2, 2), (3, 4, 2, 1)])
def test_schedule_update_statistics(dim, a, c, P):
    """Each site is the target of Binomial(s^d, 1/s^d) attempts per MCS: its
    block is active once per cycle, P cycles, k = s^d/P uniform draws."""
    n = 16 if dim == 2 else 8
    w = cw.random_small(1, dim=dim, n=n, n_cells=2, a=a, c=c, P=P)
    s = a // c
    sd = s ** dim
    per_mcs = P * c ** dim
    counts = []
    for t in range(40 if dim == 2 else 12):
        cnt = np.zeros(w.n_sites, dtype=np.int64)
        for sp in range(per_mcs):
            tg = oracle.subpass_targets(w, t, sp)
            assert len(tg) == w.n_sites // (c ** dim * P)
            np.add.at(cnt, tg, 1)
        counts.append(cnt)
    counts = np.concatenate(counts)
    assert counts.mean() == pytest.approx(1.0, abs=1e-12)  # exactly N attempts per MCS
    kmax = 6
    obs = np.array([(counts == k).sum() for k in range(kmax)] + [(counts >= kmax).sum()], dtype=float)
    pk = [math.comb(sd, k) * (1 / sd) ** k * (1 - 1 / sd) ** (sd - k) for k in range(kmax)]
    exp_ = np.array(pk + [1 - sum(pk)]) * len(counts)
    chi2 = ((obs - exp_) ** 2 / np.maximum(exp_, 1e-9)).sum()
    assert chi2 < 30.0, (obs, exp_)


def test_colour_permutations_uniform():
    w = cw.random_small(1, dim=2, n=16, n_cells=2)
    seen = {}
    for t in range(2400):
        perm = tuple(oracle.colour_perm(w, t, 0))
        assert sorted(perm) == [0, 1, 2, 3]
        seen[perm] = seen.get(perm, 0) + 1
    assert len(seen) == 24
    obs = np.array(list(seen.values()), dtype=float)
    chi2 = ((obs - 100.0) ** 2 / 100.0).sum()
    assert chi2 < 60.0  # 23 degrees of freedom


def test_replay_is_splittable():
    """Advancing by n1 then n2 sub-passes equals advancing by n1 + n2."""
    w = cw.random_small(3, dim=2, n=16, n_cells=5, act=True, perimeter=True)
    s1 = oracle.State(w)
    s2 = oracle.State(w)
    s1.replay_subpasses(13)
    s2.replay_subpasses(5)
    s2.replay_subpasses(8)
    assert np.array_equal(s1.lattice, s2.lattice)
    assert np.array_equal(s1.act, s2.act)
    assert np.array_equal(s1.V, s2.V) and np.array_equal(s1.A, s2.A)
    assert (s1.t, s1.sp) == (s2.t, s2.sp)


def test_replay_block_subset_matches_full_subpass():
    w = cw.random_small(8, dim=3, n=8, n_cells=6, perimeter=True, act=True, a=4, c=2, P=8)
    full = oracle.State(w)
    full.replay_subpasses(3)   # now at sp == 3 of MCS 0
    part = oracle.State(w)
    part.replay_subpasses(3)
    full.replay_subpasses(1)
    nblk = (w.nx // 2) * (w.ny // 2) * (w.nz // 2)
    part.replay_blocks(0, 3, 0, np.arange(nblk))
    assert np.array_equal(full.lattice, part.lattice)
    assert np.array_equal(full.V, part.V) and np.array_equal(full.A, part.A)


# ---------------------------------------------------------------------------
# the tiled schedule (tile = T > 0): tiles of edge T on a grid shifted per MCS,
# 2^d tile colours, P_T tile cycles per MCS; in an epoch the tiles of one
# colour run their share of the MCS's sub-passes while the others are dormant
# ---------------------------------------------------------------------------

def _tile_colour(coords, off, n, T):
    """Tile colour (parity of the tile coordinates) of sites (x, y, z) for a
    tile grid of edge T offset by off."""
    col = np.zeros(len(coords[0]), dtype=np.int64)
    for d, (x, o, L) in enumerate(zip(coords, off, n)):
        col += (((x - o) % L) // T % 2) << d
    return col


@pytest.mark.parametrize("dim,n,T,P,PT", [(2, 32, 8, 4, 1), (2, 32, 8, 4, 2), (3, 16, 8, 8, 2)])
def test_tiled_schedule_update_statistics(dim, n, T, P, PT):
    """Per MCS: exactly s^d attempts in every block (so N in all), each site
    the target of Binomial(s^d, 1/s^d) of them; every epoch's attempts lie in
    tiles of one colour, each colour taking P_T epochs per MCS; the grid
    offset is a multiple of a, uniform below T along each axis."""
    a, c = 4, 2
    s = a // c
    sd = s ** dim
    w = cw.random_small(2, dim=dim, n=n, n_cells=3, a=a, c=c, P=P).replace(tile=T, tile_cycles=PT)
    st = oracle.State(w)
    epochs = PT * 2 ** dim
    n_mcs = 60 if dim == 2 else 16
    shape = (w.nx, w.ny, w.nz)
    counts = []
    for t in range(n_mcs):
        tg = st.replay_trace(epochs)
        assert len(tg) == w.n_sites
        cnt = np.bincount(tg, minlength=w.n_sites)
        counts.append(cnt)
        x, y, z = tg % w.nx, (tg // w.nx) % w.ny, tg // (w.nx * w.ny)
        blk = x // s + (w.nx // s) * (y // s + (w.ny // s) * (z // s))
        assert (np.bincount(blk, minlength=w.n_sites // sd) == sd).all()
        off = oracle.tile_offset(w, t)
        cols = _tile_colour((x, y, z)[:dim], off[:dim], shape[:dim], T).reshape(epochs, -1)
        seen = []
        for e in range(epochs):
            assert len(np.unique(cols[e])) == 1, "epoch %d of MCS %d spans tile colours" % (e, t)
            seen.append(int(cols[e][0]))
        assert sorted(seen) == sorted(list(range(2 ** dim)) * PT)
    counts = np.concatenate(counts)
    kmax = min(sd, 5)
    obs = np.array([(counts == k).sum() for k in range(kmax)] + [(counts >= kmax).sum()], dtype=float)
    pk = [math.comb(sd, k) * (1 / sd) ** k * (1 - 1 / sd) ** (sd - k) for k in range(kmax)]
    exp_ = np.array(pk + [1 - sum(pk)]) * len(counts)
    keep = exp_ > 0
    chi2 = ((obs[keep] - exp_[keep]) ** 2 / exp_[keep]).sum()
    assert chi2 < 30.0, (obs, exp_)
    offs = np.array([oracle.tile_offset(w, t)[:dim] for t in range(4000)])
    assert (offs % a == 0).all() and (offs >= 0).all() and (offs < T).all()
    for d in range(dim):
        obs = np.bincount(offs[:, d] // a, minlength=T // a).astype(float)
        chi2 = ((obs - 4000 / (T // a)) ** 2 / (4000 / (T // a))).sum()
        assert chi2 < 25.0, (d, obs)


def _cells_inside_tiles(dim, n, T, seed, act):
    """A lattice whose cells sit in the middle of the tiles of MCS 0's tile
    grid: in every tile two touching 3^d cells of random types, at least
    five sites from every tile border."""
    base = cw.random_small(seed, dim=dim, n=n, n_cells=1, edge=3, perimeter=True, act=act, a=4, c=2,
                           P=4 if dim == 2 else 8)
    off = oracle.tile_offset(base.replace(tile=T), 0)
    rng = np.random.default_rng(seed)
    lat = np.zeros((n,) * dim, dtype=np.int32)
    nt = n // T
    cid = 0
    for tc in np.ndindex(*(nt,) * dim):
        lo = [int(off[dim - 1 - k]) + tc[k] * T + T // 2 - 3 for k in range(dim)]  # (z, y, x) order
        for part in range(2):
            cid += 1
            sl = [slice(0, 0)] * dim
            for k in range(dim):
                start = lo[k] + (3 if (part and k == dim - 1) else 0)
                sl[k] = np.arange(start, start + 3) % n
            lat[np.ix_(*sl)] = cid
    ct = np.zeros(cid + 1, dtype=np.uint8)
    ct[1:] = rng.integers(1, 3, size=cid)
    actv = None
    if act:
        actv = np.where(lat > 0, rng.integers(0, 30, size=lat.shape), 0).astype(np.uint8)
    lat_ = lat if dim == 3 else lat[None]
    if actv is not None and dim == 2:
        actv = actv[None]
    vt = base.v_target.copy()
    vt[1:3] = 10 if dim == 2 else 30
    lv = base.lambda_v.copy()
    lv[1:3] = 80
    return base.replace(lattice=lat_, cell_type=ct, act=actv, v_target=vt, lambda_v=lv, T=18.0), off


@pytest.mark.parametrize("dim,n,T,PT,act", [(2, 64, 16, 1, False), (2, 64, 16, 4, True), (3, 32, 16, 1, True),
                                             (3, 32, 16, 8, False)])
def test_tiled_replay_equals_global_for_cells_inside_tiles(dim, n, T, PT, act):
    """The tiled schedule runs the global schedule's sub-passes, rounds and
    Philox draws tile by tile.  When every cell lies inside one tile, far
    from its borders, no attempt reads a site another tile changes and no
    cell's tallies change in two tiles, so one MCS of the tiled replay must
    equal one MCS of the global replay bit for bit (lattice, tallies, Act)."""
    w, off = _cells_inside_tiles(dim, n, T, 40 + dim + PT, act)
    g = oracle.State(w)
    tl = oracle.State(w.replace(tile=T, tile_cycles=PT))
    acc_g = g.replay_run(1)
    acc_t = tl.replay_run(1)
    assert acc_g > 20, "the check needs accepted copies"
    # the premise held during the MCS: no cell came within two sites of a border of MCS 0's grid
    lat = g.lattice.reshape((n,) * dim)
    for k in range(dim):
        o = int(off[dim - 1 - k])
        pos = (np.arange(n) - o) % T
        near = (pos < 2) | (pos >= T - 2)
        sl = [slice(None)] * dim
        sl[k] = near
        assert (lat[tuple(sl)] <= 0).all()
    assert acc_t == acc_g
    assert np.array_equal(tl.lattice, g.lattice)
    assert np.array_equal(tl.V, g.V) and np.array_equal(tl.A, g.A)
    if act:
        assert np.array_equal(tl.act, g.act)
