"""Composite variable tracking (Methods, "Composite variable tracking",
Eq. 10 and Eq. 11) on the GPU against the replay oracle, bit for bit.

The sweep keeps every cell's coordinate sums beside its size on each
accepted copy; the oracle's replay does the same (its tracking is pinned to
the lattice in tests/test_oracle_tracking.py).  Compared after uneven
numbers of sub-passes, so that checks fall inside MCS as well as at their
ends (where the sums are moved into bounds), with cells crossing the
periodic boundary.
"""
import numpy as np
import pytest

import cpm_workloads as cw
import oracle
from tests.test_oracle_tracking import brute_sums, drifting

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


def _cases():
    out = [("drift_2d", drifting(2, 3, False)), ("drift_2d_act", drifting(2, 4, True)),
           ("drift_3d_act", drifting(3, 5, True))]
    w = cw.random_small(11, dim=2, n=32, n_cells=12, edge=3, act=True, a=8, c=2, P=4)
    out.append(("pers_2d_a8", cw.with_motility(w, lambda_pers=40, mu=0.6, dt=2)))
    w = cw.random_small(12, dim=3, n=16, n_cells=10, edge=3, act=True, obstacles=0.04, a=8, c=2, P=16)
    out.append(("obst_3d_a8", cw.with_motility(w, chem=cw.uniform_field((16, 16, 16), 3, (0.2, 1.0, 0.5)),
                                               lambda_chem=300)))
    return out


CASES = _cases()


@pytest.mark.parametrize("name,w", CASES, ids=[c[0] for c in CASES])
def test_tracked_sums_bit_exact_with_replay(cpm, name, w):
    sim = cpm.Sim(w)
    sim.track_centroids(True)
    plain = cpm.Sim(w)
    ref = oracle.State(w, track=True)
    assert np.array_equal(sim.read_centroid_sums(), ref.csum), name
    per = ref.subpasses_per_mcs()
    for n_sub in [3, per - 3, 1, per - 1] + [per] * 10:
        sim.step_subpasses(n_sub)
        plain.step_subpasses(n_sub)
        ref.replay_subpasses(n_sub)
        lat = sim.read_lattice()
        assert np.array_equal(lat, ref.lattice), name
        assert np.array_equal(plain.read_lattice(), lat), "tracking changed the dynamics (%s)" % name
        V, A = sim.read_tallies()
        assert np.array_equal(V, ref.V) and np.array_equal(A, ref.A), name
        S = sim.read_centroid_sums()
        assert np.array_equal(S, ref.csum), (name, int(np.abs(S - ref.csum).max()))
    sim.close()
    plain.close()


def test_tracking_started_mid_run_and_after_a_load(cpm):
    w = drifting(2, 6, True)
    sim = cpm.Sim(w)
    ref = oracle.State(w)
    per = ref.subpasses_per_mcs()
    sim.step_subpasses(2 * per + 3)
    with pytest.raises(cpm.CPMError):
        sim.read_centroid_sums()
    sim.track_centroids(True)
    lat = sim.read_lattice()
    assert np.array_equal(sim.read_centroid_sums(), ref.track_sums_of(lat))
    # carried on: the sums stay those of the lattice, each site at its image nearest S / V
    sim.step_subpasses(3 * per + 1)
    lat = sim.read_lattice()
    S = sim.read_centroid_sums()
    V, _ = sim.read_tallies()
    S_b, cnt = brute_sums(w, lat, S)
    live = cnt > 0
    live[0] = False
    assert np.array_equal(V[live], cnt[live])
    assert np.array_equal(S[live], S_b[live])
    # a loaded lattice restarts the sums
    other = drifting(2, 7, True).lattice
    sim.load_lattice(other)
    assert np.array_equal(sim.read_centroid_sums(), ref.track_sums_of(other))
    sim.track_centroids(False)
    with pytest.raises(cpm.CPMError):
        sim.read_centroid_sums()
    sim.close()


def _batch_members():
    w2 = cw.random_small(22, dim=2, n=32, n_cells=14, edge=3, act=True, a=8, c=2, P=4)
    return [drifting(2, 21, True),
            cw.with_motility(w2, chem=cw.uniform_field((1, 32, 32), 2, (0.3, 1.0)), lambda_chem=300),
            drifting(2, 23, True)]


def test_tracked_sums_in_a_batch(cpm):
    """Members of uneven sizes and rounds per MCS, each bit-exact with its
    own replay, sums included; the persistent loop refuses tracking."""
    ws = _batch_members()
    b = cpm.Batch(ws)
    b.track_centroids(True)
    with pytest.raises(cpm.CPMError):
        b.set_persistent(True)
    refs = [oracle.State(w, track=True) for w in ws]
    for i, r in enumerate(refs):
        assert np.array_equal(b.read_centroid_sums(i), r.csum)
    for n in (1, 2, 3):
        b.step(n)
        for i, r in enumerate(refs):
            r.replay_run(n)
            assert np.array_equal(b.read_lattice(i), r.lattice), i
            V, A = b.read_tallies(i)
            assert np.array_equal(V, r.V) and np.array_equal(A, r.A), i
            assert np.array_equal(b.read_centroid_sums(i), r.csum), i
    b.close()


def test_batch_tracking_started_after_steps(cpm):
    ws = _batch_members()
    b = cpm.Batch(ws)
    b.step(2)
    b.track_centroids(True)
    refs = [oracle.State(w) for w in ws]
    for i, r in enumerate(refs):
        assert np.array_equal(b.read_centroid_sums(i), r.track_sums_of(b.read_lattice(i))), i
    b.step(3)
    for i, w in enumerate(ws):
        lat = b.read_lattice(i)
        S = b.read_centroid_sums(i)
        V, _ = b.read_tallies(i)
        S_b, cnt = brute_sums(w, lat, S)
        live = cnt > 0
        live[0] = False
        assert np.array_equal(V[live], cnt[live]), i
        assert np.array_equal(S[live], S_b[live]), i
    b.track_centroids(False)
    with pytest.raises(cpm.CPMError):
        b.read_centroid_sums(0)
    b.step(1)
    b.close()
