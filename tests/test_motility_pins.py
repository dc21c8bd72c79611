"""Pins of the oracle's motility terms (Eq. 4 chemotaxis, Eq. 5 to Eq. 7
persistence) against closed forms: the energy of axis and diagonal copies in
a uniform field, the retraction convention, the persistence direction after
rigid translations (also across the periodic edge) and its mu-blend, and the
drift of cells along a uniform field in the serial chain."""
import ctypes
import math

import numpy as np

import cpm_workloads as cw
import oracle


def _one_square(n=16, edge=4, x0=5, y0=6, types=(1,)):
    lat = np.zeros((1, n, n), np.int32)
    lat[0, y0:y0 + edge, x0:x0 + edge] = 1
    ct = np.array([0, types[0]], np.uint8)
    J, lv, vt, lp, at, la, ma = cw._params()
    cw._sym(J, 1, 0, 10)
    lv[1], vt[1] = 1, edge * edge
    return cw.Workload("sq", 2, n, n, 1, J, lv, vt, lp, at, la, ma, 10.0, 1, 4, 2, 4, 7, 3, lat, ct)


def _n_idx(dim, d):
    """Neighbour index whose source i = j + off gives copy direction d = j - i."""
    off = oracle.neighbour_offsets(dim)  # rows (dx, dy, dz)
    for k, o in enumerate(off):
        if tuple(-o[:dim]) == tuple(d):
            return k
    raise KeyError(d)


def test_chemotaxis_energy_closed_forms():
    w = cw.with_motility(_one_square(), chem=cw.uniform_field((1, 16, 16), 2, (1, 0)), lambda_chem=5)
    st = oracle.State(w)
    j = 6 * 16 + 9   # the first medium site right of the cell (x = 9, y = 6)
    # extension along +x: the source is the cell site left of j
    q, r = st.motility(j, _n_idx(2, (1, 0)))
    assert q == -16 * 5 and abs(r + 5.0) < 1e-12
    # diagonal copy (+1, +1): -lambda / sqrt(2)
    j2 = 10 * 16 + 9
    q, r = st.motility(j2, _n_idx(2, (1, 1)))
    assert q == math.floor(-16 * 5 / math.sqrt(2)) and abs(r + 5 / math.sqrt(2)) < 1e-12
    # retraction: medium copied into the cell's left edge moves it along +x as well (sigma_j's lambda)
    j3 = 7 * 16 + 5
    q, r = st.motility(j3, _n_idx(2, (1, 0)))
    assert q == -80 and abs(r + 5.0) < 1e-12
    # against the field: positive
    j4 = 7 * 16 + 4
    q, r = st.motility(j4, _n_idx(2, (-1, 0)))
    assert q == 80 and abs(r - 5.0) < 1e-12


def _translate(st, dx, dy):
    st.lattice[0] = np.roll(st.lattice[0], (dy, dx), axis=(0, 1))


def test_persistence_update_closed_forms():
    w = cw.with_motility(_one_square(), lambda_pers=3, mu=0.0, dt=1)
    st = oracle.State(w)                     # centroids recorded at t = 0
    X0 = st.centroids()[1]
    assert np.allclose(X0[:2], [6.5, 7.5])
    upd = lambda t: oracle.lib().orc_pers_update(ctypes.byref(st.params),  # noqa: E731
                                                 oracle._ptr(st.lattice, ctypes.c_int32), t)
    _translate(st, 2, 0)
    upd(1)
    assert np.allclose(st.pers_dir[1], [1, 0, 0])
    # across the periodic edge: 13 sites to the right is 3 to the left on a 16-site axis
    _translate(st, 0, 13)
    upd(2)
    assert np.allclose(st.pers_dir[1], [0, -1, 0])
    # mu = 0.5 blends the new unit step with the previous direction, then renormalises
    w2 = cw.with_motility(_one_square(), lambda_pers=3, mu=0.5, dt=1)
    s2 = oracle.State(w2)
    s2.pers_dir[1] = [0.0, 1.0, 0.0]
    up2 = lambda t: oracle.lib().orc_pers_update(ctypes.byref(s2.params),  # noqa: E731
                                                 oracle._ptr(s2.lattice, ctypes.c_int32), t)
    _translate(s2, 1, 0)
    up2(1)
    assert np.allclose(s2.pers_dir[1], [2 ** -0.5, 2 ** -0.5, 0])
    # no displacement: unchanged
    before = s2.pers_dir[1].copy()
    up2(2)
    assert np.array_equal(s2.pers_dir[1], before)


def test_persistence_energy_and_lookback():
    w = cw.with_motility(_one_square(), lambda_pers=4, mu=0.0, dt=2)
    st = oracle.State(w)
    upd = lambda t: oracle.lib().orc_pers_update(ctypes.byref(st.params),  # noqa: E731
                                                 oracle._ptr(st.lattice, ctypes.c_int32), t)
    _translate(st, 0, 1)
    upd(1)                                   # t - dt < t0: nothing yet
    assert np.array_equal(st.pers_dir[1], [0, 0, 0])
    _translate(st, 0, 1)
    upd(2)                                   # displacement over 2 MCS: (0, 2)
    assert np.allclose(st.pers_dir[1], [0, 1, 0])
    j = (6 + 2 + 4) * 16 + 6                 # medium site above the moved cell
    q, r = st.motility(j, _n_idx(2, (0, 1)))
    assert q == -64 and abs(r + 4.0) < 1e-12


def test_serial_chain_drifts_along_the_field():
    """Eight cells in a uniform +x field, lambda_chem = 20 (T = 20): after 200
    MCS every track has moved to +x, on average by several sites, and not
    along y."""
    w = cw.random_small(5, dim=2, n=48, n_cells=8, edge=4, perimeter=False)
    w = cw.with_motility(w, chem=cw.uniform_field((1, 48, 48), 2, (1, 0)), lambda_chem=20)
    st = oracle.State(w)
    X0 = st.centroids()
    disp = np.zeros((w.n_cells + 1, 3))
    prev = X0
    for _ in range(20):
        st.serial_run(10)
        X = st.centroids()
        d = X - prev
        d[:, 0] -= 48 * np.round(d[:, 0] / 48)
        d[:, 1] -= 48 * np.round(d[:, 1] / 48)
        disp += np.nan_to_num(d)
        prev = X
    dx, dy = disp[1:, 0], disp[1:, 1]
    assert dx.mean() > 5 and dx.mean() > 3 * abs(dy.mean()), (dx, dy)
