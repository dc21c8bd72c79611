"""Cell sorting by differential adhesion (Results, Fig. 4): the parallel
scheme against the serial CPM (oracle (a)).

Two cell types in a confluent 128x128 tissue (cpm_workloads.sorting_2d)
sort themselves; the kinetics are measured, as in the paper, by the share of
heterotypic interfaces among all cell-cell interfaces (Moore pairs) over
time.  Sixteen seeds of the serial chain and sixteen of the GPU scheme, with the
paper's setting of 4x4 areas and a 2x2 checkerboard (one colour cycle per
MCS) and with larger 8x8 areas; the paper reports that the checkerboard
setting does not change sorting (Supplementary, sorting accuracy).

Bound per time point: |mean GPU - mean serial| <= max(0.015, 4 x the
standard error of the difference).  The test also requires that sorting
happens (the heterotypic share falls by at least 0.15 in the serial chain
over 3,000 MCS).
"""
import multiprocessing as mp
from concurrent.futures import ProcessPoolExecutor

import numpy as np
import pytest

import cpm_workloads as cw

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

SEEDS = list(range(1, 17))
TIMES = [0, 10, 100, 300, 1000, 3000]


def hetero_fraction(lat, cell_type):
    g = np.asarray(lat)[0]
    het = tot = 0
    for dy, dx in ((0, 1), (1, -1), (1, 0), (1, 1)):  # each unordered Moore pair once
        nb = np.roll(g, (-dy, -dx), axis=(0, 1))
        m = (g > 0) & (nb > 0) & (g != nb)
        tot += int(m.sum())
        het += int((m & (cell_type[g] != cell_type[nb])).sum())
    return het / tot


def run_serial(seed):
    import oracle
    w = cw.sorting_2d(seed)
    st = oracle.State(w)
    out, t = [], 0
    for T in TIMES:
        st.serial_run(T - t)
        t = T
        out.append(hetero_fraction(st.lattice, w.cell_type))
    return out


@pytest.fixture(scope="module")
def serial():
    ctx = mp.get_context("spawn")
    with ProcessPoolExecutor(max_workers=min(16, mp.cpu_count()), mp_context=ctx) as ex:
        return np.array(list(ex.map(run_serial, SEEDS)))


@pytest.fixture(scope="module")
def cpm():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2312_09317_gb300 import build as B
    B.build()
    from paper_2312_09317_gb300 import cpm as m
    m.load()
    return m


def run_gpu(cpm, seed, a, P):
    w = cw.sorting_2d(seed, a=a, c=2, P=P)
    sim = cpm.Sim(w)
    out, t = [], 0
    for T in TIMES:
        sim.step(T - t)
        t = T
        out.append(hetero_fraction(sim.read_lattice(), w.cell_type))
    sim.close()
    return out


@pytest.mark.parametrize("a,P", [(4, 1), (8, 4)])
def test_sorting_kinetics_match_the_serial_chain(cpm, serial, a, P):
    gpu = np.array([run_gpu(cpm, s, a, P) for s in SEEDS])
    gm, sm = gpu.mean(0), serial.mean(0)
    se = np.sqrt(gpu.var(0, ddof=1) / len(SEEDS) + serial.var(0, ddof=1) / len(SEEDS))
    print("a=%d P=%d  t=%s\n gpu    %s\n serial %s\n se     %s" % (a, P, TIMES, np.round(gm, 4), np.round(sm, 4),
                                                                np.round(se, 4)))
    assert sm[0] - sm[-1] >= 0.15, sm
    assert np.all(np.abs(gm - sm) <= np.maximum(0.015, 4 * se)), (gm, sm, se)
