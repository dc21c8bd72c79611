"""Batched ensembles against the replay oracle, bit for bit.

A batch advances many independent lattices with shared launches; each lattice
must come out exactly as the replay of the parallel scheme (and so exactly as
a single handle) after every call, including lattices with different numbers
of rounds per MCS (area edges 4 and 8) that finish their rounds at different
batch steps.
"""
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


def _check(batch, refs, tag):
    for k, ref in enumerate(refs):
        assert np.array_equal(batch.read_lattice(k), ref.lattice), "%s lattice %d" % (tag, k)
        V, A = batch.read_tallies(k)
        assert np.array_equal(V, ref.V) and np.array_equal(A, ref.A), "%s tallies %d" % (tag, k)
        if ref.act is not None:
            assert np.array_equal(batch.read_act(k), ref.act), "%s act %d" % (tag, k)
        st = batch.stats(k)
        assert st["accepts"] == ref.accepts and st["mcs"] == ref.t, "%s stats %d" % (tag, k)


def _mixed_2d():
    ws = []
    for k in range(10):
        n = [16, 24, 32, 40, 48][k % 5]
        a = 8 if k % 3 == 0 and n % 8 == 0 else 4
        ws.append(cw.random_small(100 + k, dim=2, n=n, n_cells=4 + k, edge=3, perimeter=bool(k % 2),
                                  act=bool(k % 3 == 1), obstacles=0.04 * (k % 2), a=a, c=2,
                                  P=[1, 2, 4][k % 3] if a == 4 else 4))
    return ws


def test_batch_2d_mixed_bit_exact(cpm):
    ws = _mixed_2d()
    batch = cpm.Batch(ws)
    refs = [oracle.State(w) for w in ws]
    for n in (1, 2, 3):
        batch.step(n)
        for r in refs:
            r.replay_run(n)
        _check(batch, refs, "2d after +%d" % n)
    batch.close()


def test_batch_3d_mixed_bit_exact(cpm):
    ws = [cw.random_small(200 + k, dim=3, n=[12, 16, 24][k % 3], n_cells=6 + k, edge=3, perimeter=True,
                          act=bool(k % 2), obstacles=0.03 * (k % 2), a=4, c=2, P=[1, 8][k % 2]) for k in range(6)]
    ws.append(cw.random_small(210, dim=3, n=16, n_cells=8, edge=4, perimeter=True, act=True, a=8, c=2, P=64))
    batch = cpm.Batch(ws)
    refs = [oracle.State(w) for w in ws]
    for n in (1, 2):
        batch.step(n)
        for r in refs:
            r.replay_run(n)
        _check(batch, refs, "3d after +%d" % n)
    batch.close()


def test_batch_of_the_ensemble_workload(cpm):
    """Ten members of the parameter-sweep ensemble (its recipe with small
    edges), bit-exact after 3 MCS; the Act stamps cross a clamp at MCS 0."""
    ws = cw.ensemble(10, seed=5, dim=2, side2=(32, 96), cells=(4, 40))
    batch = cpm.Batch(ws)
    refs = [oracle.State(w) for w in ws]
    batch.step(3)
    for r in refs:
        r.replay_run(3)
    _check(batch, refs, "ensemble")
    batch.close()


def test_batch_rejects_mixed_dimensions(cpm):
    ws = [cw.random_small(1, dim=2, n=16, n_cells=3), cw.random_small(2, dim=3, n=12, n_cells=3)]
    with pytest.raises(cpm.CPMError):
        cpm.Batch(ws)


def test_batch_autotune_keeps_results_exact(cpm):
    """The autotuner runs every candidate CTA shape on the batch itself; the
    members must still follow the replay exactly (3D: 7 shapes x 2 passes)."""
    ws = [cw.random_small(300 + k, dim=3, n=[16, 24][k % 2], n_cells=6 + k, edge=3, perimeter=True,
                          act=bool(k % 2), a=4, c=2, P=8) for k in range(4)]
    batch = cpm.Batch(ws)
    refs = [oracle.State(w) for w in ws]
    batch.step(1)
    choice = batch.autotune(1)
    assert 0 <= choice < 7
    batch.step(2)
    for r in refs:
        r.replay_run(1 + 7 * 2 + 2)
    _check(batch, refs, "after autotune")
    batch.close()


# ---------------------------------------------------------------------------
# the persistent loop: one cooperative launch per step, grid barriers between
# the phases of each MCS
# ---------------------------------------------------------------------------

def test_persistent_loop_bit_exact_2d_and_3d(cpm):
    """Mixed members (different rounds per MCS, Act, obstacles) advanced by
    the persistent loop match the replay after every call, across an Act
    stamp clamp (MCS 0 and 64) and with a switch between the two loops."""
    for ws, steps in ((_mixed_2d(), (1, 3, 62, 2)),
                      ([cw.random_small(400 + k, dim=3, n=[12, 16][k % 2], n_cells=5 + k, edge=3, perimeter=True,
                                        act=bool(k % 2), obstacles=0.03, a=4, c=2, P=[1, 8][k % 2])
                        for k in range(4)], (1, 2))):
        batch = cpm.Batch(ws)
        batch.set_persistent(True)
        refs = [oracle.State(w) for w in ws]
        for k, n in enumerate(steps):
            if k == len(steps) - 1:
                batch.set_persistent(False)  # the graph loop continues where the persistent one stopped
            batch.step(n)
            for r in refs:
                r.replay_run(n)
            _check(batch, refs, "persistent %dD after +%d" % (ws[0].dim, n))
        batch.close()


def test_persistent_loop_barrier_timeout_is_reported(cpm):
    """The test mode of the persistent loop makes its first CTA leave before
    the first barrier, an arrival that never comes: the other CTAs' bounded
    waits (10,000 polls) run out, the step returns CPM_E_STATE with the
    timeout message, nothing hangs, and the device stays usable for a new
    batch."""
    ws = [cw.random_small(500 + k, dim=2, n=32, n_cells=6, a=4, c=2, P=1) for k in range(8)]
    batch = cpm.Batch(ws)
    assert batch.lib.cpm_batch_set_persistent(batch.b, 2, 10000) == cpm.CPM_OK
    with pytest.raises(cpm.CPMError) as exc:
        batch.step(1)
    assert exc.value.code == cpm.CPM_E_STATE and "timed out" in str(exc.value)
    batch.close()
    fresh = cpm.Batch(ws[:2])
    fresh.set_persistent(True)
    refs = [oracle.State(w) for w in ws[:2]]
    fresh.step(2)
    for r in refs:
        r.replay_run(2)
    _check(fresh, refs, "after a timed-out batch")
    fresh.close()
