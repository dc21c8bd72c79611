"""cpm_step_noalloc, the entry point for callers that cannot allocate device
memory, against the ordinary handle-based path.

Such callers (a host framework that owns the GPU's memory budget, code that
must not allocate while it runs) pass their own lattice and tally buffers;
the call keeps its scratch in a fixed device array instead of allocating.
Its results must equal cpm_step_subpasses on a handle, bit for bit (integer
work), on two calls in a row: the second call finds the first call's
leftovers in the shared scratch and must not be affected by them.

This file is collected last so that a run stopping at the first failure has
run every other test before it; it passes alone and after the others.
"""
import ctypes

import numpy as np
import pytest

import cpm_workloads as cw

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


CASES = [
    ("3d_perim", lambda: cw.cube_cells_3d(seed=5, n=32, a=4, c=2, P=8), 3),
    ("2d_points_200", lambda: cw.point_cells_2d(seed=2, n=200, a=4, c=2, P=1), 8),
    ("3d_obstacles_a8", lambda: cw.random_small(21, dim=3, n=16, n_cells=10, edge=4, perimeter=True,
                                                obstacles=0.05, a=8, c=2, P=2, T=30.0), 5),
]


@pytest.mark.parametrize("name,factory,n_sub", CASES, ids=[c[0] for c in CASES])
def test_noalloc_matches_handle_path_twice(cpm, name, factory, n_sub):
    w = factory()
    lib = cpm.load()
    ref = cpm.Sim(w)                      # the existing entry points
    keep = []
    cfg = cpm.make_config(w, keep)
    dev = torch.device("cuda")
    lat = torch.from_numpy(np.ascontiguousarray(w.lattice, dtype=np.int32)).to(dev)
    V0, A0 = ref.read_tallies()
    V = torch.from_numpy(V0).to(dev)
    A = torch.from_numpy(A0).to(dev)
    ct = torch.from_numpy(np.ascontiguousarray(w.cell_type, dtype=np.uint8)).to(dev)
    stream = torch.cuda.current_stream()
    t, sp = 0, 0
    per_mcs = w.P * w.c ** w.dim
    for call in range(2):
        acc = ctypes.c_int64(-1)
        rc = lib.cpm_step_noalloc(ctypes.byref(cfg), lat.data_ptr(), V.data_ptr(), A.data_ptr(), ct.data_ptr(),
                                  t, sp, n_sub, ctypes.c_void_p(stream.cuda_stream), ctypes.byref(acc))
        assert rc == cpm.CPM_OK, rc
        before = ref.stats()["accepts"]
        ref.step_subpasses(n_sub)
        sp += n_sub
        t += sp // per_mcs
        sp %= per_mcs
        torch.cuda.synchronize()
        lat_ref = ref.read_lattice()
        Vr, Ar = ref.read_tallies()
        assert np.array_equal(lat.cpu().numpy(), lat_ref), "lattice, call %d" % call
        assert np.array_equal(V.cpu().numpy(), Vr), "V, call %d" % call
        assert np.array_equal(A.cpu().numpy(), Ar), "A, call %d" % call
        assert acc.value == ref.stats()["accepts"] - before, "accepts, call %d" % call
    ref.close()


def test_noalloc_matches_the_replay_oracle_from_mid_mcs(cpm):
    """Against the CPU replay of the parallel scheme directly: a 2D lattice
    with 6x6 areas (3x3 blocks, 9 rounds per colour visit: an odd count, so
    the current tallies end in the scratch's second buffer), started at
    sub-pass 3 of MCS 0 and advanced by two calls of 5 sub-passes each."""
    import oracle
    w = cw.random_small(31, dim=2, n=48, n_cells=14, edge=4, perimeter=True, obstacles=0.03, a=6, c=2, P=1,
                        T=25.0)
    st = oracle.State(w)
    st.replay_subpasses(3)
    lib = cpm.load()
    keep = []
    cfg = cpm.make_config(w, keep)
    dev = torch.device("cuda")
    lat = torch.from_numpy(st.lattice.copy()).to(dev)
    V = torch.from_numpy(st.V.copy()).to(dev)
    A = torch.from_numpy(st.A.copy()).to(dev)
    ct = torch.from_numpy(np.ascontiguousarray(w.cell_type, dtype=np.uint8)).to(dev)
    stream = torch.cuda.current_stream()
    for call in range(2):
        t, sp = st.t, st.sp
        acc = ctypes.c_int64(-1)
        rc = lib.cpm_step_noalloc(ctypes.byref(cfg), lat.data_ptr(), V.data_ptr(), A.data_ptr(), ct.data_ptr(),
                                  t, sp, 5, ctypes.c_void_p(stream.cuda_stream), ctypes.byref(acc))
        assert rc == cpm.CPM_OK, rc
        n_acc = st.replay_subpasses(5)
        torch.cuda.synchronize()
        assert np.array_equal(lat.cpu().numpy(), st.lattice), "lattice, call %d" % call
        assert np.array_equal(V.cpu().numpy(), st.V), "V, call %d" % call
        assert np.array_equal(A.cpu().numpy(), st.A), "A, call %d" % call
        assert acc.value == n_acc, "accepts, call %d" % call


def test_noalloc_refuses_a_capturing_stream(cpm):
    """The call uploads its tables from host buffers that the next call
    rewrites, so it refuses a stream under graph capture (CPM_E_INVALID)
    before it queues any work."""
    w = cw.point_cells_2d(seed=3, n=16, n_cells=4, a=4)
    lib = cpm.load()
    keep = []
    cfg = cpm.make_config(w, keep)
    dev = torch.device("cuda")
    lat = torch.from_numpy(np.ascontiguousarray(w.lattice, dtype=np.int32)).to(dev)
    V = torch.zeros(w.n_cells + 1, dtype=torch.int32, device=dev)
    ct = torch.from_numpy(np.ascontiguousarray(w.cell_type, dtype=np.uint8)).to(dev)
    x = torch.zeros(4, device=dev)
    side = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=side):
        rc = lib.cpm_step_noalloc(ctypes.byref(cfg), lat.data_ptr(), V.data_ptr(), V.data_ptr(), ct.data_ptr(),
                                  0, 0, 1, ctypes.c_void_p(side.cuda_stream), None)
        x += 1
    assert rc == cpm.CPM_E_INVALID
    g.replay()
    torch.cuda.synchronize()
    assert float(x.sum()) == 4.0


def test_noalloc_rejects_sizes_beyond_its_scratch(cpm):
    lib = cpm.load()
    dummy = torch.zeros(16, dtype=torch.int32, device="cuda")
    # 256^3 with a = 2... : 128^3 / 8 > 262,144 active blocks per round
    w = cw.point_cells_2d(seed=1, n=8, n_cells=2, a=4)
    keep = []
    cfg = cpm.make_config(w, keep)
    cfg.dim, cfg.nx, cfg.ny, cfg.nz = 3, 1024, 1024, 512
    p = dummy.data_ptr()
    assert lib.cpm_step_noalloc(ctypes.byref(cfg), p, p, p, p, 0, 0, 1, None, None) == cpm.CPM_E_LIMIT
    cfg.dim, cfg.nx, cfg.ny, cfg.nz = 2, 8, 8, 1
    cfg.n_cells = 70000
    assert lib.cpm_step_noalloc(ctypes.byref(cfg), p, p, p, p, 0, 0, 1, None, None) == cpm.CPM_E_LIMIT
    cfg.n_cells = 2
    cfg.temperature = 500.0
    assert lib.cpm_step_noalloc(ctypes.byref(cfg), p, p, p, p, 0, 0, 1, None, None) == cpm.CPM_E_LIMIT
    cfg.temperature = 20.0
    cfg.lambda_act[1] = 10
    assert lib.cpm_step_noalloc(ctypes.byref(cfg), p, p, p, p, 0, 0, 1, None, None) == cpm.CPM_E_LIMIT
    cfg.lambda_act[1] = 0
    # 2048^3 sites with 64^3 areas: few active blocks, but more than 2^31 sites
    cfg.dim, cfg.nx, cfg.ny, cfg.nz, cfg.a, cfg.c, cfg.P = 3, 2048, 2048, 2048, 64, 2, 8
    assert lib.cpm_step_noalloc(ctypes.byref(cfg), p, p, p, p, 0, 0, 1, None, None) == cpm.CPM_E_INVALID
