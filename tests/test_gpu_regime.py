"""Bit-exact parity in the regimes the benchmark times.

* The 3D Act fibre tissue at 128^3 in the schedule bench.py times for the
  1024^3 tissue, after the growth burn-in the bench runs first (60 MCS): the
  GPU's grown state (lattice, Act values, tallies, position) is handed to the
  CPU replay of the parallel scheme, and both advance 2 more MCS, compared in
  full after each.  Cells are at their target volume and the Act early
  decision fires on grown, polarised cells here.
* The 3D cube-cell model (256^3, 26-neighbourhood, perimeter) at its full
  size, compared in full after one MCS.
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


def _compare(sim, ref, tag):
    lat = sim.read_lattice()
    V, A = sim.read_tallies()
    assert np.array_equal(lat, ref.lattice), "lattice %s: %d sites differ" % (tag, int((lat != ref.lattice).sum()))
    assert np.array_equal(V, ref.V), "V %s" % tag
    assert np.array_equal(A, ref.A), "A %s" % tag
    if ref.act is not None:
        act = sim.read_act()
        assert np.array_equal(act, ref.act), "Act %s: %d differ" % (tag, int((act != ref.act).sum()))


def test_tissue_128_after_growth_bit_exact(cpm):
    w = cw.fibre_tissue_3d(seed=2, n=128, device="cuda", **cw.TISSUE_SCHEDULE)
    sim = cpm.Sim(w)
    burn = cw.TISSUE_BURN_IN
    sim.step(burn)
    st = sim.stats()
    assert st["mcs"] == burn and st["subpass"] == 0
    V, A = sim.read_tallies()
    live = V[1:] > 0
    # the grown regime: cells at their target volume (800)
    assert abs(V[1:][live].mean() - 800) < 5
    ref = oracle.State(w.replace(lattice=sim.read_lattice(), act=sim.read_act()), recount=False)
    ref.V[:] = V
    ref.A[:] = A
    ref.t = burn
    for m in range(2):
        acc0 = sim.stats()["accepts"]
        sim.step(1)
        n_acc = ref.replay_run(1)
        assert sim.stats()["accepts"] - acc0 == n_acc
        assert n_acc > 10000
        _compare(sim, ref, "tissue 128^3, MCS %d after the burn-in" % m)
    assert sim.verify() == 0
    sim.close()


def test_cube_cells_256_full_size_one_mcs(cpm):
    w = cw.cube_cells_3d(seed=1, n=256, a=4, c=2, P=8)
    sim = cpm.Sim(w)
    ref = oracle.State(w)
    sim.step(1)
    n_acc = ref.replay_run(1)
    assert sim.stats()["accepts"] == n_acc and n_acc > 0
    _compare(sim, ref, "cube cells 256^3 after MCS 0")
    sim.close()
