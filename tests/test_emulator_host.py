"""Host side of the emulator without a GPU: the oracle's summary statistics
on observation arrays with closed-form answers, the emulator's inputs, and
the statistic order shared by the library and the oracle."""
import numpy as np

import cpm_workloads as cw
from oracle import observe as oobs
from paper_2312_09317_gb300 import emulator as em


def _rows(S1, n, C, nx=64):
    cells = np.zeros((S1, n, C + 1, 12), dtype=np.int64)
    cells[:, :, 0, 0] = -1
    member = np.zeros((S1, n, 2), dtype=np.int64)
    return cells, member


def test_statistics_of_cells_in_uniform_motion():
    """Cells of 10 sites moving 3 sites in x and 4 in y every 10 MCS across the
    periodic edge: MSD = (5 lag / 10)^2, speed 0.5, unit directional
    autocorrelation, straightness 1, no arrest; fixed second moments give
    elongation 2; tallies give the volume, interface and contact statistics."""
    S1, n, C, nx, ny, every = 31, 2, 3, 64, 48, 10
    cells, member = _rows(S1, n, C)
    for s in range(S1):
        for k in range(n):
            for c in range(C):
                x = (5 + 20 * c + 3 * s) % nx
                y = (7 + 9 * k + 4 * s) % ny
                r = cells[s, k, c + 1]
                r[0] = y * nx + x
                r[1] = 10
                r[5] = 12 + c  # interface count
                r[6], r[7], r[9] = 40, 10, 0  # cxx = 4, cyy = 1, cxy = 0 about the anchor
            member[s, k] = [6, 1000 * s + 7 * k]
    out = oobs.summary_statistics(cells, member, C, (nx, ny), 20.0, 13.0, every, nx * ny)
    st = dict(zip(oobs.SUMMARY_STATS, out.T))
    np.testing.assert_allclose(st["vol_mean"], 0.5)
    np.testing.assert_allclose(st["vol_sd"], 0.0, atol=1e-12)
    np.testing.assert_allclose(st["perim_mean"], 1.0)
    np.testing.assert_allclose(st["perim_sd"], np.std([12, 13, 14]) / 13.0)
    np.testing.assert_allclose(st["msd10"], 25.0)
    np.testing.assert_allclose(st["msd50"], 625.0)
    np.testing.assert_allclose(st["msd200"], 10000.0)
    np.testing.assert_allclose(st["speed_mean"], 0.5)
    np.testing.assert_allclose(st["speed_sd"], 0.0, atol=1e-12)
    np.testing.assert_allclose(st["dac50"], 1.0)
    np.testing.assert_allclose(st["persistence"], every * (0.5 + 20))
    np.testing.assert_allclose(st["arrest"], 0.0)
    np.testing.assert_allclose(st["acceptance"], 1000.0 / (every * nx * ny))
    # sum of interface counts 39 = 2 cc + cm with cm = 6 -> cc = 16.5 -> 16.5 / 22.5
    np.testing.assert_allclose(st["contact_cc"], 16.5 / 22.5)
    np.testing.assert_allclose(st["straightness"], 1.0)
    np.testing.assert_allclose(st["elongation"], 2.0)


def test_statistics_of_resting_cells_and_a_vanished_cell():
    """Still cells: zero MSD and speed, full arrest; a cell that vanishes in
    the window leaves the tracks but its live snapshots count for volume."""
    S1, n, C, nx = 31, 1, 2, 32
    cells, member = _rows(S1, n, C)
    for s in range(S1):
        cells[s, 0, 1, :2] = [100, 8]
        cells[s, 0, 1, 6:8] = [8, 8]
        if s < 10:
            cells[s, 0, 2, :2] = [300, 4]
            cells[s, 0, 2, 6:8] = [4, 4]
        else:
            cells[s, 0, 2, 0] = -1
    out = oobs.summary_statistics(cells, member, C, (nx, nx), 8.0, 10.0, 10, nx * nx)
    st = dict(zip(oobs.SUMMARY_STATS, out[0]))
    assert st["msd10"] == 0.0 and st["speed_mean"] == 0.0 and st["arrest"] == 1.0
    np.testing.assert_allclose(st["vol_mean"], (31 * 8 + 10 * 4) / 41 / 8.0)
    np.testing.assert_allclose(st["elongation"], 1.0)


def test_statistics_scaled_by_a_zero_target_are_nan():
    """Without a perimeter constraint (A_t = 0) the interface statistics
    scaled by A_t are undefined: NaN, with no division warning; the volume
    statistics are unaffected."""
    import warnings
    S1, n, C, nx = 11, 1, 2, 32
    cells, member = _rows(S1, n, C)
    for s in range(S1):
        for c in range(C):
            cells[s, 0, c + 1, :2] = [100 + 40 * c, 8]
            cells[s, 0, c + 1, 5] = 12
            cells[s, 0, c + 1, 6:8] = [8, 8]
    with warnings.catch_warnings():
        warnings.simplefilter("error")
        out = oobs.summary_statistics(cells, member, C, (nx, nx), 8.0, 0.0, 10, nx * nx)
    st = dict(zip(oobs.SUMMARY_STATS, out[0]))
    assert np.isnan(st["perim_mean"]) and np.isnan(st["perim_sd"])
    np.testing.assert_allclose(st["vol_mean"], 1.0)


def test_sweep_points_are_on_the_simulated_grid_and_span_the_ranges():
    X = cw.sweep_points(200, 3)
    assert X.shape == (200, 7)
    for j, k in enumerate(cw.EMULATOR_PARAMS):
        lo, hi = cw.SWEEP_RANGES[k]
        assert lo - 0.05 <= X[:, j].min() and X[:, j].max() <= hi + 0.05
        assert X[:, j].max() - X[:, j].min() > 0.9 * (hi - lo)
    assert np.allclose(X[:, :4] * 10, np.round(X[:, :4] * 10))
    w = cw.emulator_run(X[0], 5)
    assert w.n_cells == cw.EMULATOR_CELLS and w.nx == cw.EMULATOR_SIDE
    assert w.J[1, 1] == int(round(X[0, 0] * 10)) and w.max_act[1] == int(X[0, 5])
    s = cw.scale_inputs(X)
    assert s.min() >= -0.01 and s.max() <= 1.01


def test_mlp_init_layout():
    p = cw.mlp_init(4, 3, [7, 16, 5])
    assert p.shape == (3, 7 * 16 + 16 + 16 * 5 + 5)
    assert not np.allclose(p[0], p[1])
    assert np.all(p[0, 112:128] == 0) and np.all(p[0, -5:] == 0)


def test_statistic_order_matches_the_library():
    assert em.STATS == oobs.SUMMARY_STATS
    assert set(em.LOG_STATS) <= set(em.STATS)


def test_invalid_network_shapes_are_rejected_without_a_gpu():
    """cpm_mlp_create validates the shape before touching the device and
    reports why through cpm_mlp_last_error(NULL)."""
    import ctypes
    from paper_2312_09317_gb300 import build as B
    from paper_2312_09317_gb300 import cpm
    B.build()
    lib = cpm.load()
    init = np.zeros(1 << 16, dtype=np.float32)
    for shape in [cpm.MlpShape(0, 7, 256, 4, 16, 1024),     # no members
                  cpm.MlpShape(5, 7, 250, 4, 16, 1024),     # width not a multiple of 8
                  cpm.MlpShape(5, 7, 256, 16, 16, 1024),    # too many layers
                  cpm.MlpShape(5, 7, 256, 4, 16, 1 << 23)]:  # too many rows
        h = ctypes.c_void_p()
        rc = lib.cpm_mlp_create(ctypes.byref(shape), init.ctypes.data_as(ctypes.c_void_p), None, ctypes.byref(h))
        assert rc == -1 and not h.value
        assert b"invalid shape" in lib.cpm_mlp_last_error(None)
    h = ctypes.c_void_p()
    assert lib.cpm_mlp_create(None, None, None, ctypes.byref(h)) == -1
    assert b"required" in lib.cpm_mlp_last_error(None)
