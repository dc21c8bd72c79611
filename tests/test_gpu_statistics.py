"""Statistical parity of the GPU sweep with the serial CPM (oracle (a)) on the
2D workload (200x200, Moore-8, 100 cells, V_t = 100).

The GPU path equals the parallel-scheme replay bit for bit; this test
measures what the parallel scheme itself changes relative to the serial
Markov chain, as the paper does for its own scheme (Results, Fig. 3-5):
64 seeds, 200 MCS of growth, then 40 snapshots 10 MCS apart; cell volume
mean and variance, interface-count mean, acceptance rate, and the mean
squared displacement of cell centroids over 10 and 50 MCS
(tests/tissue_stats.py reduces both sides).

* Large areas with frequent switching, as the paper recommends (Results,
  "Aligning the lattice update statistics"): areas of 40x40 sites, 2x2
  checkerboard, one round per colour visit (P = 400).  Every statistic's
  mean per-seed difference (both runs of a seed start from the same lattice)
  is within 2% of the serial chain's mean; its standard error is at most
  about 0.7% (variance and MSD over 50 MCS), so the bar is about three
  standard errors wide.  (Areas of 20x20
  come out at +1.4% volume variance and +1.8% MSD over 50 MCS, too close to
  the bar; 10x10 at +13% variance.)
* The paper's sorting setting (4x4 areas, 2x2 checkerboard, one cycle): the
  mean volume still matches within 2%, and the deviations of the fluctuation
  statistics that several concurrent attempts on one cell inside a round
  cause are checked to be present (variance and acceptance far above the
  serial chain's), as recorded in the design notes.
"""
import multiprocessing as mp
from concurrent.futures import ProcessPoolExecutor

import numpy as np
import pytest

import cpm_workloads as cw
from tests import tissue_stats as ts

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

SEEDS = list(range(1, 65))
BURN, SNAPS, EVERY = 200, 40, 10
TOL = 0.02


def run_serial(seed):
    import torch as th
    th.set_num_threads(1)
    import oracle
    w = cw.point_cells_2d(seed=seed)  # the schedule does not enter the serial chain
    st = oracle.State(w)
    st.serial_run(BURN)
    shape = (1, w.ny, w.nx)
    rec = ts.Recorder(shape, w.n_cells)
    rec.snapshot(th.from_numpy(st.lattice.reshape(shape)))
    acc = 0
    for _ in range(SNAPS):
        acc += st.serial_run(EVERY)
        rec.snapshot(th.from_numpy(st.lattice.reshape(shape)), st.V, st.A)
    return rec.summary(acc, w.n_sites)


def run_gpu(cpm, a, P):
    """All seeds as one batch (each member is exactly its single-lattice run)."""
    ws = [cw.point_cells_2d(seed=s, a=a, c=2, P=P) for s in SEEDS]
    b = cpm.Batch(ws)
    b.step(BURN)
    shape = (1, ws[0].ny, ws[0].nx)
    recs = [ts.Recorder(shape, w.n_cells) for w in ws]
    lat = torch.empty(shape, dtype=torch.int32, device="cuda")
    for k, r in enumerate(recs):
        b.read_lattice(k, lat)
        r.snapshot(lat)
    acc0 = [b.stats(k)["accepts"] for k in range(len(ws))]
    for _ in range(SNAPS):
        b.step(EVERY)
        for k, r in enumerate(recs):
            b.read_lattice(k, lat)
            V, A = b.read_tallies(k)
            r.snapshot(lat, V, A)
    out = [r.summary(b.stats(k)["accepts"] - acc0[k], ws[k].n_sites) for k, r in enumerate(recs)]
    b.close()
    return {k: np.array([o[k] for o in out]) for k in ts.STATS}


@pytest.fixture(scope="module")
def serial_stats():
    assert ts.EVERY == EVERY
    # the pool is started with spawn, independent of the GPU context
    ctx = mp.get_context("spawn")
    with ProcessPoolExecutor(max_workers=min(16, mp.cpu_count()), mp_context=ctx) as ex:
        res = list(ex.map(run_serial, SEEDS))
    return {k: np.array([r[k] for r in res]) for k in ts.STATS}


@pytest.fixture(scope="module")
def cpm():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2312_09317_gb300 import build as B
    B.build()
    from paper_2312_09317_gb300 import cpm as m
    m.load()
    return m


def _report(g, s):
    """Per statistic: the means, and the mean of the per-seed difference GPU - serial
    (both runs of a seed start from the same lattice) relative to the serial mean, with
    its standard error."""
    out = {}
    for k in ts.STATS:
        d = (g[k] - s[k]) / abs(s[k].mean())
        out[k] = dict(gpu=round(float(g[k].mean()), 6), serial=round(float(s[k].mean()), 6),
                      rel=round(float(d.mean()), 5), se_rel=round(float(d.std(ddof=1) / np.sqrt(len(d))), 5))
    return out


def test_statistics_match_serial_with_large_areas_frequent_switching(cpm, serial_stats):
    g = run_gpu(cpm, 40, 400)
    rep = _report(g, serial_stats)
    print("a=40, P=400:", rep)
    for k in ts.STATS:
        assert abs(rep[k]["rel"]) <= TOL, (k, rep)


def test_statistics_with_the_papers_4x4_areas(cpm, serial_stats):
    g = run_gpu(cpm, 4, 1)
    s = serial_stats
    rep = _report(g, s)
    print("a=4, P=1:", rep)
    assert abs(rep["vmean"]["rel"]) <= TOL, rep
    # the deviations of the 4x4 / 2x2 setting (in-round concurrency on one cell)
    assert rep["vvar"]["rel"] > 0.5, rep
    assert rep["acc"]["rel"] > 0.2, rep
    assert rep["amean"]["rel"] > 0.02, rep
