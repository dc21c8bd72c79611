"""Pins of the emulator's FP64 oracle (``oracle.mlp``, ``oracle.observe``)
against facts that do not come from the oracle itself: textbook values of the
normal CDF, central finite differences of the loss, the least-squares
optimum of a linear model (numpy's lstsq), closed forms of Adam's first
steps, and lattice geometry whose counts follow from the neighbourhood.
"""
import itertools
import math

import numpy as np
import pytest

from oracle import mlp, observe


def _net(rng, sizes, scale=0.5):
    return [(rng.normal(0, scale, (o, i)), rng.normal(0, 0.1, o)) for i, o in zip(sizes[:-1], sizes[1:])]


def test_gelu_textbook_values():
    # GELU(z) = z Phi(z); Phi(1) = 0.8413447460685429, Phi(-1) = 0.15865525393145707,
    # Phi(2) = 0.9772498680518208 (standard normal table)
    assert mlp.gelu(0.0) == 0.0
    assert abs(mlp.gelu(1.0) - 0.8413447460685429) < 1e-15
    assert abs(mlp.gelu(-1.0) + 0.15865525393145707) < 1e-15
    assert abs(mlp.gelu(2.0) - 2 * 0.9772498680518208) < 1e-15
    assert abs(mlp.gelu(10.0) - 10.0) < 1e-12 and abs(mlp.gelu(-10.0)) < 1e-12
    # GELU'(0) = Phi(0) = 1/2; GELU'(z) -> 1 and -> 0 at the tails
    assert mlp.gelu_grad(0.0) == 0.5
    assert abs(mlp.gelu_grad(8.0) - 1.0) < 1e-12 and abs(mlp.gelu_grad(-8.0)) < 1e-12


def test_gelu_grad_matches_finite_differences():
    z = np.linspace(-6, 6, 241)
    h = 1e-6
    fd = (mlp.gelu(z + h) - mlp.gelu(z - h)) / (2 * h)
    assert np.max(np.abs(fd - mlp.gelu_grad(z))) < 1e-8


def test_backward_matches_central_differences():
    rng = np.random.default_rng(7)
    params = _net(rng, [7, 9, 8, 6, 5])
    X = rng.uniform(0, 1, (11, 7))
    Y = rng.normal(0, 1, (11, 5))
    _, grads, _ = mlp.loss_and_grads(params, X, Y)
    h = 1e-6
    worst = 0.0
    for l, (W, b) in enumerate(params):
        for arr, g in ((W, grads[l][0]), (b, grads[l][1])):
            for idx in itertools.islice(np.ndindex(arr.shape), 0, None, 3):
                old = arr[idx]
                arr[idx] = old + h
                lp = mlp.mse(mlp.forward(params, X)[0], Y)[0]
                arr[idx] = old - h
                lm = mlp.mse(mlp.forward(params, X)[0], Y)[0]
                arr[idx] = old
                fd = (lp - lm) / (2 * h)
                worst = max(worst, abs(fd - g[idx]) / max(1e-6, abs(fd) + abs(g[idx])))
    assert worst < 1e-6, worst


def test_dropped_gelu_term_is_detected_by_finite_differences():
    """A plausible slip (GELU' taken as Phi alone) must fail the check above."""
    rng = np.random.default_rng(8)
    params = _net(rng, [3, 6, 2])
    X = rng.uniform(-1, 1, (5, 3))
    Y = rng.normal(0, 1, (5, 2))
    P, (Hs, Zs) = mlp.forward(params, X)
    _, dP = mlp.mse(P, Y)
    dZ1 = (dP @ params[1][0]) * (0.5 * (1 + np.vectorize(math.erf)(Zs[0] / math.sqrt(2))))
    wrong = dZ1.T @ Hs[0]
    right = mlp.backward(params, (Hs, Zs), dP)[0][0]
    assert np.max(np.abs(wrong - right)) > 1e-4


def test_linear_model_gradient_vanishes_at_least_squares_optimum():
    """One linear layer: the MSE gradient is zero at numpy's lstsq solution
    and equals 2/(n o) R^T [X 1] at any other point (R the residual)."""
    rng = np.random.default_rng(9)
    X = rng.normal(0, 1, (40, 7))
    Y = rng.normal(0, 1, (40, 3))
    Xa = np.hstack([X, np.ones((40, 1))])
    sol, *_ = np.linalg.lstsq(Xa, Y, rcond=None)
    params = [(sol[:7].T.copy(), sol[7].copy())]
    _, grads, _ = mlp.loss_and_grads(params, X, Y)
    assert np.max(np.abs(grads[0][0])) < 1e-12 and np.max(np.abs(grads[0][1])) < 1e-12
    params = [(sol[:7].T + 0.3, sol[7] - 0.2)]
    _, grads, P = mlp.loss_and_grads(params, X, Y)
    R = P - Y
    assert np.allclose(grads[0][0], 2.0 / R.size * R.T @ X, atol=1e-13)
    assert np.allclose(grads[0][1], 2.0 / R.size * R.sum(0), atol=1e-13)


def test_adam_closed_forms():
    # eps = 0: bias correction makes every step of a constant gradient exactly lr sign(g)
    w, m, v = np.array([1.0, -2.0, 0.5]), np.zeros(3), np.zeros(3)
    g = np.array([0.3, -4.0, 1e-3])
    for t in range(1, 6):
        w_new, m, v = mlp.adam(w, g, m, v, 0.01, 0.9, 0.999, 0.0, t)
        assert np.allclose(w - w_new, 0.01 * np.sign(g), rtol=0, atol=1e-15)
        w = w_new
    # two steps by hand, g1 = 1, g2 = -1, b1 = 0.5, b2 = 0.75, lr = 1, eps = 0:
    # m1 = .5, v1 = .25, mhat = 1, vhat = 1 -> w = -1
    # m2 = .25 - .5 = -.25, v2 = .1875 + .25 = .4375; mhat = -.25/.75 = -1/3,
    # vhat = .4375/.4375 = 1 -> w = -1 + 1/3
    w, m, v = mlp.adam(np.array([0.0]), np.array([1.0]), np.zeros(1), np.zeros(1), 1.0, 0.5, 0.75, 0.0, 1)
    assert w[0] == -1.0
    w, m, v = mlp.adam(w, np.array([-1.0]), m, v, 1.0, 0.5, 0.75, 0.0, 2)
    assert abs(w[0] - (-1.0 + 1.0 / 3.0)) < 1e-15


def test_ensemble_and_fallback():
    rng = np.random.default_rng(3)
    p = _net(rng, [7, 5, 4])
    X = rng.uniform(0, 1, (6, 7))
    mean, std, _ = mlp.ensemble_predict([p, p, p], X)
    assert np.allclose(mean, mlp.forward(p, X)[0]) and np.max(std) < 1e-15
    std = np.array([[0.1, 0.2], [0.31, 0.0], [0.0, 0.61]])
    assert list(mlp.fallback_mask(std, np.array([0.1, 0.2]))) == [False, True, True]


def test_centroid_of_a_square_straddling_the_periodic_edge():
    lat = np.zeros((1, 10, 12), np.int32)
    ys, xs = [9, 0, 1], [11, 0, 1]
    for y in ys:
        for x in xs:
            lat[0, y, x] = 1
    c = observe.centroids(lat, 1)
    assert np.allclose(c[1], [0.0, 0.0, 0.0])  # centred on the corner site (0, 0)
    anchor, count, sums = observe.centroid_sums(lat, 1)
    assert anchor[1] == 0 and count[1] == 9 and list(sums[1]) == [0, 0, 0]
    lat3 = np.zeros((8, 8, 8), np.int32)
    lat3[np.ix_([7, 0], [3, 4], [6, 7])] = 2
    c3 = observe.centroids(lat3, 2)
    assert np.allclose(c3[2], [6.5, 3.5, 7.5]) and np.isnan(c3[1]).all()


def test_cell_medium_pairs_against_neighbourhood_counts():
    # an isolated 3x3 square, Moore-8: 72 neighbour slots, 40 ordered
    # cell-cell pairs inside (20 unordered: 6 horizontal, 6 vertical, 8 diagonal)
    lat = np.zeros((1, 9, 9), np.int32)
    lat[0, 2:5, 3:6] = 1
    assert observe.cell_medium_pairs(lat, 2) == 72 - 40
    # two squares touching along a column: the shared edge moves 3 + 2*2 = 7 pairs to cell-cell
    lat[0, 2:5, 6:9] = 2
    assert observe.cell_medium_pairs(lat, 2) == 2 * 32 - 2 * 7
    # a 2x2x2 cube, 26 neighbours: 8 * 26 slots, every pair of the 8 sites is adjacent (28 pairs)
    lat3 = np.zeros((6, 6, 6), np.int32)
    lat3[1:3, 1:3, 1:3] = 1
    assert observe.cell_medium_pairs(lat3, 3) == 8 * 26 - 2 * 28


def test_interface_tallies_split_into_cell_cell_and_cell_medium():
    """Sum of the per-cell interface counts = 2 x cell-cell pairs + cell-medium pairs."""
    import cpm_workloads as cw
    from tests import brute
    w = cw.random_small(11, dim=2, n=32, n_cells=9, edge=3)
    A = brute.interfaces(w, w.lattice)
    cm = observe.cell_medium_pairs(w.lattice, 2)
    g = w.lattice[0]
    cc = 0
    for dy, dx in itertools.product((-1, 0, 1), repeat=2):
        if (dy, dx) == (0, 0):
            continue
        nb = np.roll(g, (-dy, -dx), axis=(0, 1))
        cc += int(((g > 0) & (nb > 0) & (nb != g)).sum())
    assert cc % 2 == 0
    assert int(A[1:].sum()) == cc + cm


def test_cell_rows_agree_with_brute_tallies_and_a_hand_moment():
    import cpm_workloads as cw
    from tests import brute
    for dim in (2, 3):
        w = cw.random_small(21 + dim, dim=dim, n=16, n_cells=6, edge=3, obstacles=0.05)
        rows = observe.cell_rows(w.lattice, w.n_cells, dim)
        assert list(rows[0]) == [-1] + [0] * 11
        assert np.array_equal(rows[1:, 1], brute.volumes(w, w.lattice)[1:])
        assert np.array_equal(rows[1:, 5], brute.interfaces(w, w.lattice)[1:])
        a, cnt, sums = observe.centroid_sums(w.lattice, w.n_cells)
        assert np.array_equal(rows[:, 0], a) and np.array_equal(rows[:, 2:5], sums)
    # a 1 x 3 bar along x with the anchor at its left end: offsets 0, 1, 2
    lat = np.zeros((1, 8, 8), np.int32)
    lat[0, 4, 2:5] = 1
    r = observe.cell_rows(lat, 1, 2)[1]
    assert list(r[[2, 3, 6, 7, 9]]) == [3, 0, 5, 0, 0]
