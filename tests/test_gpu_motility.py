"""Chemotaxis (Eq. 4) and persistence (Eq. 5 to Eq. 7) on the GPU against
the replay oracle, bit for bit: lattice, tallies, Act values, accepts and
the persistence directions p_hat (exact doubles) after every call; then the
drift of cells in a uniform field against the serial chain."""
import numpy as np
import pytest

import cpm_workloads as cw
import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def cpm():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2312_09317_gb300 import build as B
    B.build()
    from paper_2312_09317_gb300 import cpm as m
    m.load()
    return m


def _field(w, kind):
    shape = (w.nz, w.ny, w.nx)
    if kind == "uniform":
        return cw.uniform_field(shape, w.dim, (1, 2) if w.dim == 2 else (1, 2, -2))
    return cw.circular_field(w.nx, w.ny, w.nz, w.dim)


def _cases():
    out = []
    for dim, n in ((2, 32), (3, 16)):
        base = cw.random_small(700 + dim, dim=dim, n=n, n_cells=6 if dim == 2 else 5, edge=4, perimeter=True, a=4,
                               c=2, P=4 if dim == 2 else 8, T=40.0)
        out.append(("chem_uniform_%dd" % dim, cw.with_motility(base, chem=_field(base, "uniform"), lambda_chem=30)))
        out.append(("chem_circular_%dd" % dim, cw.with_motility(base, chem=_field(base, "circular"), lambda_chem=-17)))
        out.append(("pers_%dd" % dim, cw.with_motility(base, lambda_pers=25, mu=0.8, dt=2)))
        act = cw.random_small(710 + dim, dim=dim, n=n, n_cells=5, edge=4, perimeter=True, act=True, obstacles=0.03,
                              a=4, c=2, P=2 if dim == 2 else 4, T=40.0)
        out.append(("all_%dd" % dim, cw.with_motility(act, chem=_field(act, "circular"), lambda_chem=20,
                                                      lambda_pers=15, mu=0.5, dt=3)))
    return out


CASES = _cases()


@pytest.mark.parametrize("name,w", CASES, ids=[c[0] for c in CASES])
def test_motility_bit_exact_with_replay(cpm, name, w):
    sim = cpm.Sim(w)
    ref = oracle.State(w)
    for n in (1, 2, 3):
        sim.step(n)
        ref.replay_run(n)
        assert np.array_equal(sim.read_lattice(), ref.lattice), name
        V, A = sim.read_tallies()
        assert np.array_equal(V, ref.V) and np.array_equal(A, ref.A), name
        if ref.act is not None:
            assert np.array_equal(sim.read_act(), ref.act), name
        assert sim.stats()["accepts"] == ref.accepts, name
        if w.pers_on:
            got = sim.read_persistence()
            assert np.array_equal(got, ref.pers_dir), (name, np.abs(got - ref.pers_dir).max())
    if w.pers_on:
        assert np.abs(ref.pers_dir[1:]).sum() > 0  # the directions were updated
    sim.close()


def test_chemotaxis_in_a_batch(cpm):
    ws = [w for name, w in CASES if name.startswith("chem") and w.dim == 2]
    b = cpm.Batch(ws)
    refs = [oracle.State(w) for w in ws]
    b.step(3)
    for k, r in enumerate(refs):
        r.replay_run(3)
        assert np.array_equal(b.read_lattice(k), r.lattice)
    b.close()


def test_persistence_is_rejected_where_it_is_not_built(cpm):
    w = dict(CASES)["pers_2d"]
    with pytest.raises(cpm.CPMError):
        cpm.Batch([w])
    with pytest.raises(cpm.CPMError):
        cpm.Sim(w.replace(tile=16, tile_cycles=1))


def test_drift_in_a_uniform_field_matches_the_serial_chain(cpm):
    """16 seeds of 8 cells on a 40x40 lattice in a +x field (lambda_chem =
    20, T = 20), 150 MCS: mean displacement along x of the GPU scheme (20x20
    areas, 2x2 checkerboard, 100 cycles per MCS, the setting the paper
    recommends for fidelity) and of the serial chain agree within
    20% (5 standard errors), and both are clearly positive."""
    def drift(run):
        out = []
        for seed in range(16):
            w = cw.random_small(800 + seed, dim=2, n=40, n_cells=8, edge=4, perimeter=False, a=20, c=2, P=100,
                                T=20.0)
            w = cw.with_motility(w, chem=cw.uniform_field((1, 40, 40), 2, (1, 0)), lambda_chem=20)
            out.append(run(w))
        return np.array(out)

    def track(positions_fn, step_fn, w):
        st0 = positions_fn()
        total = np.zeros(w.n_cells + 1)
        prev = st0
        for _ in range(15):
            step_fn(10)
            X = positions_fn()
            d = X[:, 0] - prev[:, 0]
            d -= 40 * np.round(d / 40)
            total += np.nan_to_num(d)
            prev = X
        return total[1:].mean()

    def run_serial(w):
        st = oracle.State(w)
        return track(st.centroids, st.serial_run, w)

    def run_gpu(w):
        sim = cpm.Sim(w)
        probe = oracle.State(w)

        def pos():
            probe.lattice[...] = sim.read_lattice()
            return probe.centroids()
        r = track(pos, sim.step, w)
        sim.close()
        return r

    g, s = drift(run_gpu), drift(run_serial)
    se = np.sqrt(g.var(ddof=1) / len(g) + s.var(ddof=1) / len(s))
    print("drift gpu %.3f serial %.3f se %.3f" % (g.mean(), s.mean(), se))
    assert s.mean() > 3 and g.mean() > 3
    assert abs(g.mean() - s.mean()) <= max(0.2 * s.mean(), 5 * se)
