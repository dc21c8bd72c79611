"""Statistical parity of the GPU sweep with the serial CPM (oracle (a)).

The GPU path equals the parallel-scheme replay bit for bit; this test measures
what the parallel scheme itself changes relative to the serial Markov chain,
as the paper does for its own scheme (Results, Fig. 3-5): 32 seeds of the 2D
workload (200x200, Moore-8, 100 cells, V_t = 100), 200 MCS of growth, then
statistics over 100 MCS sampled every 10 MCS: cell volume mean and variance,
perimeter (interface count) mean, acceptance rate, and the mean squared
displacement of cell centroids over 10 and 50 MCS.

Tolerances (relative, per statistic, over the 32-seed means):
* large areas with frequent switching, as the paper recommends (Results,
  "Aligning the lattice update statistics"): areas of 20x20 sites, 2x2
  checkerboard, 100 colour cycles per MCS (one round per visit).  The scheme
  matches the serial chain within 2% on volume mean, perimeter mean and
  acceptance, within 5% on volume variance and MSD (their 32-seed standard
  errors are 1-1.5%);
* the paper's sorting setting (4x4 areas, 2x2 checkerboard, one cycle): the
  volume mean still matches within 2%, while fluctuation statistics differ
  (several concurrent attempts on one cell inside a round); the test records
  them and bounds them loosely.
"""
import multiprocessing as mp
from concurrent.futures import ProcessPoolExecutor

import numpy as np
import pytest

import cpm_workloads as cw

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

SEEDS = list(range(1, 33))
BURN, SAMPLES, EVERY = 200, 10, 10


def centroids(lat, n_cells):
    """Periodic centroids (circular mean per axis) of every cell."""
    lat2 = lat.reshape(lat.shape[-2], lat.shape[-1])
    ids = lat2.ravel()
    m = ids > 0
    ys, xs = np.unravel_index(np.nonzero(m)[0], lat2.shape)
    out = np.zeros((n_cells + 1, 2))
    for d, (coord, L) in enumerate(((ys, lat2.shape[0]), (xs, lat2.shape[1]))):
        ang = coord * 2 * np.pi / L
        cs = np.bincount(ids[m], weights=np.cos(ang), minlength=n_cells + 1)
        sn = np.bincount(ids[m], weights=np.sin(ang), minlength=n_cells + 1)
        out[:, d] = (np.arctan2(sn, cs) % (2 * np.pi)) * L / (2 * np.pi)
    return out


def summarise(snapshots, tallies, accepts, n_sites, n_cells, shape):
    L = np.array(shape, dtype=float)
    traj = [np.zeros((n_cells + 1, 2))]
    prev = centroids(snapshots[0], n_cells)
    for s in snapshots[1:]:
        c = centroids(s, n_cells)
        d = c - prev
        d -= np.round(d / L) * L
        traj.append(traj[-1] + d)
        prev = c
    traj = np.array(traj)[:, 1:, :]
    V = np.array([t[0][1:] for t in tallies], dtype=float)
    A = np.array([t[1][1:] for t in tallies], dtype=float)
    msd10 = ((traj[1:] - traj[:-1]) ** 2).sum(-1).mean()
    msd50 = ((traj[5:] - traj[:-5]) ** 2).sum(-1).mean()
    return dict(vmean=V.mean(), vvar=V.var(), amean=A.mean(), acc=accepts / (SAMPLES * EVERY * n_sites),
                msd10=msd10, msd50=msd50)


def run_serial(args):
    seed, a = args
    import oracle
    w = cw.point_cells_2d(seed=seed, a=a, c=2, P=1)  # the schedule does not enter the serial chain
    st = oracle.State(w)
    st.serial_run(BURN)
    snaps, tall, acc = [st.lattice.copy()], [], 0
    for _ in range(SAMPLES):
        acc += st.serial_run(EVERY)
        snaps.append(st.lattice.copy())
        tall.append((st.V.copy(), st.A.copy()))
    return summarise(snaps, tall, acc, w.n_sites, w.n_cells, (w.ny, w.nx))


def run_gpu(cpm, seed, a, P):
    w = cw.point_cells_2d(seed=seed, a=a, c=2, P=P)
    sim = cpm.Sim(w)
    sim.step(BURN)
    snaps, tall = [sim.read_lattice()], []
    acc0 = sim.stats()["accepts"]
    for _ in range(SAMPLES):
        sim.step(EVERY)
        snaps.append(sim.read_lattice())
        tall.append(sim.read_tallies())
    acc = sim.stats()["accepts"] - acc0
    sim.close()
    return summarise(snaps, tall, acc, w.n_sites, w.n_cells, (w.ny, w.nx))


@pytest.fixture(scope="module")
def serial_stats():
    # the pool is started with spawn, independent of the GPU context
    ctx = mp.get_context("spawn")
    with ProcessPoolExecutor(max_workers=min(16, mp.cpu_count()), mp_context=ctx) as ex:
        res = list(ex.map(run_serial, [(s, 4) for s in SEEDS]))
    return {k: np.array([r[k] for r in res]) for k in res[0]}


@pytest.fixture(scope="module")
def cpm():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2312_09317_gb300 import build as B
    B.build()
    from paper_2312_09317_gb300 import cpm as m
    m.load()
    return m


def _gpu_stats(cpm, a, P):
    res = [run_gpu(cpm, s, a, P) for s in SEEDS]
    return {k: np.array([r[k] for r in res]) for k in res[0]}


def _rel(g, s):
    return abs(g.mean() - s.mean()) / abs(s.mean())


def test_statistics_match_serial_with_large_areas_frequent_switching(cpm, serial_stats):
    g = _gpu_stats(cpm, 20, 100)
    s = serial_stats
    report = {k: (round(float(g[k].mean()), 5), round(float(s[k].mean()), 5), round(_rel(g[k], s[k]), 4))
              for k in s}
    print("a=20, P=100 (gpu, serial, rel):", report)
    for k in ("vmean", "amean", "acc"):
        assert _rel(g[k], s[k]) <= 0.02, (k, report)
    for k in ("vvar", "msd10", "msd50"):
        assert _rel(g[k], s[k]) <= 0.05, (k, report)


def test_statistics_with_the_papers_4x4_areas(cpm, serial_stats):
    g = _gpu_stats(cpm, 4, 1)
    s = serial_stats
    report = {k: (round(float(g[k].mean()), 5), round(float(s[k].mean()), 5), round(_rel(g[k], s[k]), 4))
              for k in s}
    print("a=4 (gpu, serial, rel):", report)
    assert _rel(g["vmean"], s["vmean"]) <= 0.02, report
    # documented deviations of the 4x4/2x2 setting (in-round concurrency on one cell)
    assert g["amean"].mean() > s["amean"].mean()
    assert _rel(g["amean"], s["amean"]) <= 0.25, report
    assert _rel(g["acc"], s["acc"]) <= 1.5, report
    assert _rel(g["msd50"], s["msd50"]) <= 2.0, report
