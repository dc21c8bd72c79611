"""The C ABI library on a machine without a GPU: it builds, loads, exports every
function the headers under include/ declare, and rejects invalid configurations before
touching the device."""
import ctypes
import os
import re

import numpy as np
import pytest

import cpm_workloads as cw
from paper_2312_09317_gb300 import build as B
from paper_2312_09317_gb300 import cpm

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_functions():
    names = set()
    for f in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if f.endswith(".h"):
            src = open(os.path.join(ROOT, "include", f)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(cpm_[a-z0-9_]+)\s*\(", src))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    B.build()
    return cpm.load()


def test_header_declares_the_boundary():
    names = _declared_functions()
    for n in ("cpm_create", "cpm_step", "cpm_read_lattice", "cpm_stats", "cpm_destroy", "cpm_last_error"):
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    for n in _declared_functions():
        assert hasattr(lib, n), n
        assert n in cpm._SIGNATURES, n


def test_config_struct_layout_matches_header():
    # offsets of the last fields follow from the C layout rules
    assert ctypes.sizeof(cpm.Config) % 8 == 0
    assert cpm.Config.temperature.offset % 8 == 0
    assert cpm.Config.seed.offset % 8 == 0


def _create(w, **over):
    keep = []
    cfg = cpm.make_config(w, keep)
    for k, v in over.items():
        setattr(cfg, k, v)
    h = ctypes.c_void_p()
    rc = cpm.load().cpm_create(ctypes.byref(cfg), None, ctypes.byref(h))
    return rc, cpm.load().cpm_last_error(None).decode()


@pytest.mark.parametrize("field,value,msg", [
    ("dim", 4, "dim"),
    ("a", 6, "multiples of a"),
    ("c", 1, "c >= 2"),
    ("a", 2, "c >= 2"),
    ("P", 3, "P must divide"),
    ("temperature", 0.0, "temperature"),
    ("temperature", 1e6, "temperature"),
    ("obstacle_type", 0, "obstacle_type"),
    ("n_cells", -1, "n_cells"),
    ("n_cells", 1 << 23, "n_cells"),  # ids share the lattice word with the Act stamp: 24 bits
    ("t0", -5, "t0"),
])
def test_invalid_configs_are_rejected_without_a_gpu(lib, field, value, msg):
    w = cw.random_small(1, dim=2, n=16, n_cells=3, a=4, c=2, P=1)
    rc, err = _create(w, **{field: value})
    assert rc == cpm.CPM_E_INVALID
    assert msg in err


def test_gap_between_active_blocks_is_enforced(lib):
    # a = 4, c = 4 gives blocks of edge 1 that are 3 apart: fine; a = 3, c = 3 would be 2 apart: fine;
    # a = 2, c = 2 gives blocks 1 apart: rejected
    w = cw.random_small(1, dim=2, n=16, n_cells=3, a=2, c=2, P=1)
    rc, err = _create(w)
    assert rc == cpm.CPM_E_INVALID and "apart" in err


def test_bad_lattice_and_act_rejected(lib):
    w = cw.random_small(2, dim=2, n=16, n_cells=3, a=4, act=True)
    lat = w.lattice.copy()
    lat.flat[5] = 99
    rc, err = _create(w.replace(lattice=lat))
    assert rc == cpm.CPM_E_INVALID and "init_lattice" in err
    act = w.act.copy()
    act[w.lattice == 0] = 0
    act.flat[np.flatnonzero(w.lattice.ravel() == 0)[0]] = 3
    rc, err = _create(w.replace(act=act))
    assert rc == cpm.CPM_E_INVALID and "init_act" in err
    J = w.J.copy()
    J[1, 2] += 1
    rc, err = _create(w.replace(J=J))
    assert rc == cpm.CPM_E_INVALID and "symmetric" in err


def test_null_handle_calls_fail_cleanly(lib):
    assert lib.cpm_step(None, 1) == cpm.CPM_E_HANDLE
    assert lib.cpm_read_lattice(None, None, 0) == cpm.CPM_E_HANDLE
    assert lib.cpm_kernel_launches(None) == 0
    assert lib.cpm_track_centroids(None, 1) == cpm.CPM_E_HANDLE
    assert lib.cpm_read_centroid_sums(None, None, 0) == cpm.CPM_E_HANDLE
    lib.cpm_destroy(None)


def test_motility_settings_are_checked_without_a_gpu(lib):
    w = cw.random_small(3, dim=2, n=32, n_cells=4, a=4, c=2, P=4)
    wc = cw.with_motility(w, chem=cw.uniform_field((1, 32, 32), 2, (1, 0)), lambda_chem=5)
    rc, err = _create(wc.replace(tile=8, tile_cycles=1))
    assert rc == cpm.CPM_E_INVALID and "global schedule" in err
    wp = cw.with_motility(w, lambda_pers=5, mu=0.5, dt=0)
    rc, err = _create(wp)
    assert rc == cpm.CPM_E_INVALID and "dt_pers" in err
    wp = cw.with_motility(w, lambda_pers=5, mu=1.5, dt=2)
    rc, err = _create(wp)
    assert rc == cpm.CPM_E_INVALID and "mu_pers" in err


def test_create_errors_are_per_thread(lib):
    """cpm_last_error(NULL) reports the calling thread's own failed create,
    even when another thread fails in between."""
    import threading
    w = cw.random_small(1, dim=2, n=16, n_cells=3, a=4, c=2, P=1)
    gate = threading.Barrier(2)
    seen = {}

    def worker(name, field, value):
        keep = []
        c = cpm.make_config(w, keep)
        setattr(c, field, value)
        h = ctypes.c_void_p()
        rc = lib.cpm_create(ctypes.byref(c), None, ctypes.byref(h))
        gate.wait()  # both creates have failed before either message is read
        seen[name] = (rc, lib.cpm_last_error(None).decode())

    ts = [threading.Thread(target=worker, args=("dim", "dim", 4)),
          threading.Thread(target=worker, args=("temp", "temperature", 0.0))]
    for t in ts:
        t.start()
    for t in ts:
        t.join()
    assert seen["dim"][0] == cpm.CPM_E_INVALID and "dim" in seen["dim"][1]
    assert seen["temp"][0] == cpm.CPM_E_INVALID and "temperature" in seen["temp"][1]
