"""GPU sweep against the CPU replay oracle of the parallel scheme, bit for bit.

Every case runs the CUDA library through its C ABI and oracle (b) side by
side on the same seeded input and compares, after every MCS (or sub-pass),
the lattice, the volume and interface tallies, the Act values and the number
of accepted copies.  Integer work, so the bar is exact equality.
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


def _compare(sim, ref, tag=""):
    lat = sim.read_lattice()
    V, A = sim.read_tallies()
    assert np.array_equal(lat, ref.lattice), "lattice %s: %d sites differ" % (tag, int((lat != ref.lattice).sum()))
    assert np.array_equal(V, ref.V), "V %s" % tag
    assert np.array_equal(A, ref.A), "A %s" % tag
    if ref.act is not None:
        act = sim.read_act()
        assert np.array_equal(act, ref.act), "Act %s: %d differ" % (tag, int((act != ref.act).sum()))
    assert sim.stats()["accepts"] == ref.accepts, tag


CASES = [
    # (name, workload factory, MCS)
    ("2d_adh_vol", lambda: cw.random_small(1, dim=2, n=20, n_cells=8, perimeter=False, a=4, c=2, P=1), 6),
    ("2d_perim", lambda: cw.random_small(2, dim=2, n=24, n_cells=10, perimeter=True, a=4, c=2, P=4), 6),
    ("2d_act_obst", lambda: cw.random_small(3, dim=2, n=28, n_cells=12, perimeter=True, act=True,
                                            obstacles=0.08, a=4, c=2, P=2), 6),
    ("2d_a8_c2", lambda: cw.random_small(4, dim=2, n=32, n_cells=10, edge=5, perimeter=True, act=True,
                                         a=8, c=2, P=1), 4),
    ("2d_a9_c3", lambda: cw.random_small(5, dim=2, n=27, n_cells=9, edge=4, perimeter=True, a=9, c=3, P=3), 4),
    ("2d_3types_hotT", lambda: cw.random_small(6, dim=2, n=20, n_cells=12, perimeter=True, act=True,
                                               n_types=3, T=200.0, a=4, c=2, P=1), 5),
    ("3d_adh_vol", lambda: cw.random_small(7, dim=3, n=12, n_cells=8, perimeter=False, a=4, c=2, P=8), 3),
    ("3d_perim", lambda: cw.random_small(8, dim=3, n=12, n_cells=10, perimeter=True, a=4, c=2, P=1), 3),
    ("3d_act_obst", lambda: cw.random_small(9, dim=3, n=16, n_cells=12, perimeter=True, act=True,
                                            obstacles=0.05, a=8, c=2, P=64), 2),
    ("3d_a8_P2", lambda: cw.random_small(10, dim=3, n=16, n_cells=10, edge=4, perimeter=True, act=True,
                                         a=8, c=2, P=2), 2),
    # larger 3D lattices; 44 and 52 give CTA bricks (8 x 4 x 4 active blocks) that overhang the active grid
    ("3d_staged_adh_vol", lambda: cw.random_small(41, dim=3, n=48, n_cells=40, edge=5, perimeter=False,
                                                  a=4, c=2, P=8), 2),
    ("3d_staged_act_obst", lambda: cw.random_small(42, dim=3, n=48, n_cells=40, edge=5, perimeter=True, act=True,
                                                   obstacles=0.05, a=4, c=2, P=1), 2),
    ("3d_staged_ragged44", lambda: cw.random_small(43, dim=3, n=44, n_cells=30, edge=5, perimeter=True, act=True,
                                                   a=4, c=2, P=2), 2),
    ("3d_staged_ragged52", lambda: cw.random_small(44, dim=3, n=52, n_cells=30, edge=5, perimeter=True,
                                                   obstacles=0.03, a=4, c=2, P=8), 2),
]


@pytest.mark.parametrize("name,factory,n_mcs", CASES, ids=[c[0] for c in CASES])
def test_bit_exact_against_replay(cpm, name, factory, n_mcs):
    w = factory()
    sim = cpm.Sim(w, stream=torch.cuda.current_stream())
    ref = oracle.State(w)
    _compare(sim, ref, "initial")
    for m in range(n_mcs):
        sim.step(1)
        ref.replay_run(1)
        _compare(sim, ref, "after MCS %d" % m)
    assert sim.verify() == 0
    sim.close()


def test_non_cubic_lattice(cpm):
    """Extents that differ per axis (ragged number of active blocks per CTA)."""
    w = cw.cube_cells_3d(seed=3, n=24, a=4, c=2, P=8)
    lat = np.zeros((8, 12, 20), dtype=np.int32)
    lat[:] = w.lattice[:8, :12, :20]
    ids = np.unique(lat[lat > 0])
    remap = np.zeros(w.n_cells + 1, dtype=np.int32)
    remap[ids] = np.arange(1, len(ids) + 1)
    lat = np.where(lat > 0, remap[np.maximum(lat, 0)], lat).astype(np.int32)
    ct = np.ones(len(ids) + 1, dtype=np.uint8)
    ct[0] = 0
    w2 = w.replace(nx=20, ny=12, nz=8, lattice=lat, cell_type=ct)
    sim = cpm.Sim(w2)
    ref = oracle.State(w2)
    for m in range(3):
        sim.step(1)
        ref.replay_run(1)
        _compare(sim, ref, "MCS %d" % m)


def test_subpass_granularity_and_splitting(cpm):
    w = cw.random_small(12, dim=2, n=24, n_cells=9, perimeter=True, act=True, a=4, c=2, P=2)
    sim = cpm.Sim(w)
    ref = oracle.State(w)
    for n in (1, 3, 2, 7, 11):
        sim.step_subpasses(n)
        ref.replay_subpasses(n)
        _compare(sim, ref, "after %d more sub-passes" % n)
    st = sim.stats()
    assert (st["mcs"], st["subpass"]) == (ref.t, ref.sp)


def test_step_splits_like_one_call(cpm):
    w = cw.random_small(13, dim=3, n=12, n_cells=8, perimeter=True, act=True, a=4, c=2, P=8)
    s1 = cpm.Sim(w)
    s2 = cpm.Sim(w)
    s1.step(5)
    s2.step(2)
    s2.step(3)
    assert np.array_equal(s1.read_lattice(), s2.read_lattice())
    assert np.array_equal(s1.read_act(), s2.read_act())
    V1, A1 = s1.read_tallies()
    V2, A2 = s2.read_tallies()
    assert np.array_equal(V1, V2) and np.array_equal(A1, A2)


def test_act_stamps_survive_many_mcs(cpm):
    """Over 200 MCS the uint8 stamps wrap and are clamped every 64 MCS; Act
    values must still equal the oracle's explicit decay."""
    w = cw.random_small(14, dim=2, n=16, n_cells=4, edge=4, perimeter=True, act=True, a=4, c=2, P=1)
    w.max_act[1:3] = [127, 9]
    mx = w.max_act[w.cell_type[np.maximum(w.lattice, 0)]]
    w = w.replace(act=np.where(w.lattice > 0, np.minimum(w.act, mx), 0).astype(np.uint8))
    sim = cpm.Sim(w)
    ref = oracle.State(w)
    for chunk in (63, 1, 1, 70, 65):
        sim.step(chunk)
        ref.replay_run(chunk)
        _compare(sim, ref, "at MCS %d" % ref.t)


def test_empty_and_degenerate_lattices(cpm):
    # all medium: nothing can happen
    w = cw.random_small(15, dim=2, n=16, n_cells=1, perimeter=True)
    w = w.replace(lattice=np.zeros_like(w.lattice), cell_type=np.zeros(1, dtype=np.uint8))
    sim = cpm.Sim(w)
    sim.step(3)
    assert sim.stats()["accepts"] == 0
    assert not sim.read_lattice().any()
    # one cell filling everything, plus obstacles: nothing can change either
    lat = np.ones_like(w.lattice)
    lat.flat[::7] = -1
    w1 = w.replace(lattice=lat, cell_type=np.array([0, 1], dtype=np.uint8))
    sim = cpm.Sim(w1)
    sim.step(2)
    assert sim.stats()["accepts"] == 0
    assert np.array_equal(sim.read_lattice(), lat)
    # single-pixel cells must never vanish
    w2 = cw.point_cells_2d(seed=3, n=40, n_cells=30, a=4, c=2, P=1)
    w2.v_target[1] = 1
    w2.lambda_v[1] = 1
    sim = cpm.Sim(w2)
    ref = oracle.State(w2)
    sim.step(5)
    ref.replay_run(5)
    _compare(sim, ref, "tiny cells")
    V, _ = sim.read_tallies()
    assert np.all(V[1:] >= 1)


def test_point_cells_200_full_size_bit_exact(cpm):
    """The 200x200 2D workload as specified (Moore-8, 100 cells, V_t = 100),
    bit-exact over 20 MCS."""
    w = cw.point_cells_2d(seed=1)
    sim = cpm.Sim(w)
    ref = oracle.State(w)
    for m in range(20):
        sim.step(1)
        ref.replay_run(1)
    _compare(sim, ref, "200^2 point cells after 20 MCS")


def test_load_lattice_resets_tallies(cpm):
    w = cw.random_small(16, dim=2, n=16, n_cells=5, perimeter=True)
    sim = cpm.Sim(w)
    sim.step(2)
    lat = sim.read_lattice()
    sim.load_lattice(lat)
    assert sim.verify() == 0
    d = torch.from_numpy(lat).cuda()
    sim.load_lattice(d)
    out = torch.empty_like(d)
    sim.read_lattice(out)
    assert torch.equal(out, d)


def test_tissue_64_bit_exact(cpm):
    """The tissue workload (fibre obstacles, Act, perimeter, 26-neighbourhood)
    at 64^3, bit-exact after every MCS."""
    w = cw.fibre_tissue_3d(seed=2, n=64, a=4, c=2, P=8, device="cuda")
    assert (w.lattice < 0).mean() > 0.1
    sim = cpm.Sim(w)
    ref = oracle.State(w)
    for m in range(3):
        sim.step(1)
        ref.replay_run(1)
        _compare(sim, ref, "tissue 64^3 after MCS %d" % m)
    assert sim.verify() == 0


def test_tissue_1024_sampled(cpm):
    """1024^3 tissue workload in the launch configuration bench.py times: the
    areas of cpm_workloads.TISSUE_SCHEDULE (the same grid of active blocks and
    CTAs), with one round per sub-pass so that a single round can be replayed
    for sampled blocks.  After 2 MCS and 3 sub-passes,
    one more round runs on the GPU; the oracle replays that round for 4,096
    sampled active blocks from the GPU's state before it, and their sites and
    Act values must match.  Tallies are checked at full size by a device
    recount, obstacles by comparison with the input."""
    a, c = cw.TISSUE_SCHEDULE["a"], cw.TISSUE_SCHEDULE["c"]
    w = cw.fibre_tissue_3d(seed=1, n=1024, device="cuda", a=a, c=c, P=(a // c) ** 3)
    assert (w.a // w.c) ** 3 // w.P == 1  # one round per sub-pass: the sampled round is the whole sub-pass
    sim = cpm.Sim(w)
    sim.step(2)
    sim.step_subpasses(3)
    st = sim.stats()
    t, sp = st["mcs"], st["subpass"]
    assert sp == 3
    pre_lat = sim.read_lattice()
    pre_act = sim.read_act()
    V, A = sim.read_tallies()
    sim.step_subpasses(1)
    post_lat = sim.read_lattice()
    post_act = sim.read_act()
    assert sim.verify() == 0
    assert np.array_equal(post_lat < 0, w.lattice < 0)

    ref = oracle.State(w.replace(lattice=pre_lat, act=pre_act), recount=False)
    ref.V[:] = V
    ref.A[:] = A
    s = w.a // w.c
    C = w.c ** 3
    col = oracle.colour_perm(w, t, sp // C)[sp % C]
    cx, cy, cz = col % w.c, (col // w.c) % w.c, col // (w.c * w.c)
    nb = w.nx // s
    rng = np.random.default_rng(7)
    k = 4096
    bx = rng.integers(0, nb // w.c, k) * w.c + cx
    by = rng.integers(0, nb // w.c, k) * w.c + cy
    bz = rng.integers(0, nb // w.c, k) * w.c + cz
    blocks = np.unique(bx + nb * (by + nb * bz))
    ref.replay_blocks(t, sp, 0, blocks)
    bxs, bys, bzs = blocks % nb, (blocks // nb) % nb, blocks // (nb * nb)
    for dz in range(s):
        for dy in range(s):
            for dx in range(s):
                z, y, x = bzs * s + dz, bys * s + dy, bxs * s + dx
                assert np.array_equal(post_lat[z, y, x], ref.lattice[z, y, x])
                assert np.array_equal(post_act[z, y, x], ref.act[z, y, x])
    changed = int((pre_lat != post_lat).sum())
    assert changed > 0
    sim.close()


TILE_CASES = [
    ("2d_T8_PT1", lambda: cw.random_small(31, dim=2, n=32, n_cells=10, perimeter=True, a=4, c=2, P=4)
     .replace(tile=8, tile_cycles=1), 4),
    ("2d_T8_PT4_act_obst", lambda: cw.random_small(32, dim=2, n=32, n_cells=12, perimeter=True, act=True,
                                                   obstacles=0.06, a=4, c=2, P=4).replace(tile=8, tile_cycles=4), 4),
    ("2d_T16_PT2_a8", lambda: cw.random_small(33, dim=2, n=64, n_cells=16, edge=5, perimeter=True, act=True,
                                              a=8, c=2, P=2).replace(tile=16, tile_cycles=2), 3),
    ("3d_T8_PT1", lambda: cw.random_small(34, dim=3, n=16, n_cells=10, perimeter=True, a=4, c=2, P=8)
     .replace(tile=8, tile_cycles=1), 2),
    ("3d_T8_PT2_act_obst", lambda: cw.random_small(35, dim=3, n=16, n_cells=12, perimeter=True, act=True,
                                                   obstacles=0.05, a=4, c=2, P=8).replace(tile=8, tile_cycles=2), 2),
    ("3d_tissue_T16", lambda: cw.fibre_tissue_3d(seed=3, n=64, a=4, c=2, P=8, device="cuda")
     .replace(tile=16, tile_cycles=1), 2),
    ("3d_cubes_T24", lambda: cw.cube_cells_3d(seed=4, n=96, a=4, c=2, P=8).replace(tile=24, tile_cycles=2), 2),
]


@pytest.mark.parametrize("name,factory,n_mcs", TILE_CASES, ids=[c[0] for c in TILE_CASES])
def test_tiled_schedule_bit_exact(cpm, name, factory, n_mcs):
    w = factory()
    sim = cpm.Sim(w)
    ref = oracle.State(w)
    for m in range(n_mcs):
        sim.step(1)
        ref.replay_run(1)
        _compare(sim, ref, "tiled %s after MCS %d" % (name, m))
    # finer steps: single epochs
    for n in (1, 2, 3):
        sim.step_subpasses(n)
        ref.replay_subpasses(n)
        _compare(sim, ref, "tiled %s after %d more epochs" % (name, n))
    st = sim.stats()
    assert (st["mcs"], st["subpass"]) == (ref.t, ref.sp)
    assert st["attempts"] == ref.t * w.n_sites + ref.sp * w.n_sites // ref.subpasses_per_mcs()
    assert sim.verify() == 0
    sim.close()
