"""CPU oracle for the cellular Potts model sweep: test infrastructure only.

Only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` may import this package.  It shares
no code with the CUDA library; the two meet only in the seeded inputs of
``cpm_workloads``.

The arithmetic lives in ``cpm_oracle.c`` (plain C, compiled with gcc by
``build()``); this module marshals numpy arrays into it with ctypes.

* ``serial_run``  -- oracle (a): the serial CPM chain (Methods, Eq. 1, Eq. 2,
  Eq. 3, Eq. 8, Eq. 9) in double precision with exact exp.
* ``replay_run``  -- oracle (b): replay of the parallel checkerboard scheme
  (Results, Fig. 2A/B, Fig. 3A/B) with Philox counters, integer energies and
  the integer threshold table.
* ``replay_blocks`` -- one round of (b) restricted to a list of blocks, for
  sampled checks.
* ``State(w, track=True)`` -- (b) with composite variable tracking (Eq. 10,
  Eq. 11): per-cell coordinate sums in ``State.csum``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "cpm_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "libcpm_oracle.so")

MAXT = 8


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no fused multiply-add contraction, so the
    table arithmetic rounds the same way on every machine)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".%d.tmp" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


class Params(ctypes.Structure):
    _fields_ = [
        ("dim", ctypes.c_int32), ("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("nz", ctypes.c_int32),
        ("J", (ctypes.c_int32 * MAXT) * MAXT),
        ("lambda_v", ctypes.c_int32 * MAXT), ("v_target", ctypes.c_int32 * MAXT),
        ("lambda_p", ctypes.c_int32 * MAXT), ("a_target", ctypes.c_int32 * MAXT),
        ("lambda_act", ctypes.c_int32 * MAXT), ("max_act", ctypes.c_int32 * MAXT),
        ("T", ctypes.c_double),
        ("obstacle_type", ctypes.c_int32),
        ("a", ctypes.c_int32), ("c", ctypes.c_int32), ("P", ctypes.c_int32),
        ("seed", ctypes.c_uint64),
        ("n_cells", ctypes.c_int32),
        ("cell_type", ctypes.POINTER(ctypes.c_uint8)),
        ("tile", ctypes.c_int32),
        ("tile_cycles", ctypes.c_int32),
        ("chem_field", ctypes.POINTER(ctypes.c_int16)),
        ("lambda_chem", ctypes.c_int32 * MAXT),
        ("lambda_pers", ctypes.c_int32 * MAXT),
        ("mu_pers", ctypes.c_double * MAXT),
        ("dt_pers", ctypes.c_int32 * MAXT),
        ("pers_dir", ctypes.POINTER(ctypes.c_double)),
        ("pers_hist", ctypes.POINTER(ctypes.c_double)),
        ("pers_hist_len", ctypes.c_int32),
        ("pers_t0", ctypes.c_int64),
        ("csum", ctypes.POINTER(ctypes.c_int64)),
    ]


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        P = ctypes.POINTER
        i32p, u8p, i64p, u32p = P(ctypes.c_int32), P(ctypes.c_uint8), P(ctypes.c_int64), P(ctypes.c_uint32)
        _lib.orc_philox4x32_10.argtypes = [u32p, u32p, u32p]
        _lib.orc_serial_run.argtypes = [P(Params), i32p, u8p, i32p, i32p, ctypes.c_int64,
                                        P(ctypes.c_uint64), i64p, i64p]
        f64p = P(ctypes.c_double)
        _lib.orc_motility.argtypes = [P(Params), i32p, ctypes.c_int64, ctypes.c_int, i64p, f64p]
        _lib.orc_centroids.argtypes = [P(Params), i32p, f64p]
        _lib.orc_centroids.restype = None
        _lib.orc_pers_update.argtypes = [P(Params), i32p, ctypes.c_int64]
        _lib.orc_pers_update.restype = None
        _lib.orc_replay_run.argtypes = [P(Params), i32p, u8p, i32p, i32p, i64p, i32p, ctypes.c_int64, i64p]
        _lib.orc_replay_round.argtypes = [P(Params), i32p, u8p, i32p, i32p, ctypes.c_int64, ctypes.c_int32,
                                          ctypes.c_int32, i64p, ctypes.c_int64, i64p]
        _lib.orc_recount.argtypes = [P(Params), i32p, i32p, i32p]
        _lib.orc_recount.restype = None
        _lib.orc_delta_h.argtypes = [P(Params), i32p, u8p, i32p, i32p, ctypes.c_int64, ctypes.c_int,
                                     i64p, i64p, P(ctypes.c_double), i64p, i64p, P(ctypes.c_double),
                                     P(ctypes.c_double)]
        _lib.orc_colour_perm.argtypes = [P(Params), ctypes.c_int64, ctypes.c_int, i32p]
        _lib.orc_thr_table.argtypes = [ctypes.c_double, u32p, ctypes.c_int64]
        _lib.orc_thr_table.restype = ctypes.c_int64
        _lib.orc_ln_table.argtypes = [i32p]
        _lib.orc_ln_table.restype = None
        _lib.orc_expq_size.restype = ctypes.c_int32
        _lib.orc_expq_table.argtypes = [i32p, ctypes.c_int32]
        _lib.orc_expq_table.restype = None
        _lib.orc_xoshiro_seed.argtypes = [ctypes.c_uint64, P(ctypes.c_uint64)]
        _lib.orc_xoshiro_seed.restype = None
        _lib.orc_neighbour_offsets.argtypes = [ctypes.c_int, i32p]
        _lib.orc_subpass_targets.argtypes = [P(Params), ctypes.c_int64, ctypes.c_int32, i64p]
        _lib.orc_subpass_targets.restype = ctypes.c_int64
        _lib.orc_replay_trace.argtypes = [P(Params), i32p, u8p, i32p, i32p, i64p, i32p, ctypes.c_int64, i64p,
                                          i64p, ctypes.c_int64, i64p]
        _lib.orc_tile_offset_of.argtypes = [P(Params), ctypes.c_int64, i64p]
        _lib.orc_tile_offset_of.restype = None
        _lib.orc_track_init.argtypes = [P(Params), i32p, i32p, i64p]
        _lib.orc_track_init.restype = None
        _lib.orc_track_rewrap.argtypes = [P(Params), i32p, i64p]
        _lib.orc_track_rewrap.restype = None
    return _lib


def _ptr(a, ct):
    return a.ctypes.data_as(ctypes.POINTER(ct)) if a is not None else None


class State:
    """Oracle state for one workload: lattice, Act values, tallies, position.
    Keeps a reference to every array handed to C."""

    def __init__(self, w, act_on=None, recount=True, track=False):
        self.w = w
        self.lattice = np.ascontiguousarray(w.lattice, dtype=np.int32).copy()
        self.cell_type = np.ascontiguousarray(w.cell_type, dtype=np.uint8).copy()
        act_on = w.act_on if act_on is None else act_on
        if act_on:
            self.act = (np.zeros_like(self.lattice, dtype=np.uint8) if w.act is None
                        else np.ascontiguousarray(w.act, dtype=np.uint8).copy())
        else:
            self.act = None
        self.chem = (np.ascontiguousarray(w.chem_field, dtype=np.int16).copy()
                     if getattr(w, "chem_field", None) is not None else None)
        pers = getattr(w, "pers_on", False)
        self.pers_len = int(np.max(w.dt_pers)) + 1 if pers else 0
        self.pers_dir = np.zeros((w.n_cells + 1, 3)) if pers else None
        self.pers_hist = np.full((max(self.pers_len, 1), w.n_cells + 1, 3), np.nan) if pers else None
        self.params = make_params(w, self.cell_type, self)
        self.V = np.zeros(w.n_cells + 1, dtype=np.int32)
        self.A = np.zeros(w.n_cells + 1, dtype=np.int32)
        if recount:
            lib().orc_recount(ctypes.byref(self.params), _ptr(self.lattice, ctypes.c_int32),
                              _ptr(self.V, ctypes.c_int32), _ptr(self.A, ctypes.c_int32))
        self.t = 0
        self.sp = 0
        # composite variable tracking (Eq. 11): per-cell coordinate sums, centroid = S / V
        self.csum = None
        if track:
            self.csum = np.zeros((w.n_cells + 1, 3), dtype=np.int64)
            self.params.csum = _ptr(self.csum, ctypes.c_int64)
            lib().orc_track_init(ctypes.byref(self.params), _ptr(self.lattice, ctypes.c_int32),
                                 _ptr(self.V, ctypes.c_int32), _ptr(self.csum, ctypes.c_int64))
        if pers:  # the centroids at the start: the first look-back point
            lib().orc_pers_update(ctypes.byref(self.params), _ptr(self.lattice, ctypes.c_int32), 0)
        self.rng = (ctypes.c_uint64 * 4)()
        lib().orc_xoshiro_seed(ctypes.c_uint64(w.seed), self.rng)
        self.accepts = 0

    # ----------------------------------------------------------------
    def serial_run(self, n_mcs: int) -> int:
        acc = ctypes.c_int64(0)
        t = ctypes.c_int64(self.t)
        rc = lib().orc_serial_run(ctypes.byref(self.params), _ptr(self.lattice, ctypes.c_int32),
                                  _ptr(self.act, ctypes.c_uint8), _ptr(self.V, ctypes.c_int32),
                                  _ptr(self.A, ctypes.c_int32), n_mcs, self.rng, ctypes.byref(t),
                                  ctypes.byref(acc))
        if rc != 0:
            raise RuntimeError("orc_serial_run failed: %d" % rc)
        self.t = t.value
        self.accepts += acc.value
        return acc.value

    def replay_subpasses(self, n_sub: int) -> int:
        t = ctypes.c_int64(self.t)
        sp = ctypes.c_int32(self.sp)
        acc = ctypes.c_int64(0)
        rc = lib().orc_replay_run(ctypes.byref(self.params), _ptr(self.lattice, ctypes.c_int32),
                                  _ptr(self.act, ctypes.c_uint8), _ptr(self.V, ctypes.c_int32),
                                  _ptr(self.A, ctypes.c_int32), ctypes.byref(t), ctypes.byref(sp),
                                  n_sub, ctypes.byref(acc))
        if rc != 0:
            raise RuntimeError("orc_replay_run failed: %d" % rc)
        self.t, self.sp = t.value, sp.value
        self.accepts += acc.value
        return acc.value

    def replay_trace(self, n_sub: int) -> np.ndarray:
        """replay_subpasses, returning the target site of every attempt in
        the order the replay makes them (early rejects included)."""
        t = ctypes.c_int64(self.t)
        sp = ctypes.c_int32(self.sp)
        acc = ctypes.c_int64(0)
        n = ctypes.c_int64(0)
        cap = int(n_sub) * self.w.n_sites // max(1, self.subpasses_per_mcs()) + self.w.n_sites
        buf = np.zeros(cap, dtype=np.int64)
        rc = lib().orc_replay_trace(ctypes.byref(self.params), _ptr(self.lattice, ctypes.c_int32),
                                    _ptr(self.act, ctypes.c_uint8), _ptr(self.V, ctypes.c_int32),
                                    _ptr(self.A, ctypes.c_int32), ctypes.byref(t), ctypes.byref(sp),
                                    n_sub, ctypes.byref(acc), _ptr(buf, ctypes.c_int64), cap, ctypes.byref(n))
        if rc != 0 or n.value > cap:
            raise RuntimeError("orc_replay_trace failed: %d (%d attempts, room for %d)" % (rc, n.value, cap))
        self.t, self.sp = t.value, sp.value
        self.accepts += acc.value
        return buf[:n.value].copy()

    def subpasses_per_mcs(self) -> int:
        """Schedule units per MCS: sub-passes (global rounds) or epochs (tiled)."""
        if getattr(self.w, "tile", 0):
            return self.w.tile_cycles * 2 ** self.w.dim
        return self.w.P * self.w.c ** self.w.dim

    def replay_run(self, n_mcs: int) -> int:
        return self.replay_subpasses(n_mcs * self.subpasses_per_mcs())

    def replay_blocks(self, t: int, sp: int, r: int, blocks) -> int:
        """Round r of sub-pass sp of MCS t restricted to ``blocks`` (no Act
        decay here); tallies are read from this state's V and A."""
        blk = np.ascontiguousarray(blocks, dtype=np.int64)
        acc = ctypes.c_int64(0)
        rc = lib().orc_replay_round(ctypes.byref(self.params), _ptr(self.lattice, ctypes.c_int32),
                                    _ptr(self.act, ctypes.c_uint8), _ptr(self.V, ctypes.c_int32),
                                    _ptr(self.A, ctypes.c_int32), t, sp, r, _ptr(blk, ctypes.c_int64),
                                    len(blk), ctypes.byref(acc))
        if rc != 0:
            raise RuntimeError("orc_replay_round failed: %d" % rc)
        return acc.value

    def motility(self, j: int, n_idx: int):
        """Motility terms of the copy from neighbour n_idx of j into j: (Q4 as
        the replay applies them, real as the serial chain does)."""
        q, r = ctypes.c_int64(0), ctypes.c_double(0.0)
        lib().orc_motility(ctypes.byref(self.params), _ptr(self.lattice, ctypes.c_int32), j, n_idx,
                           ctypes.byref(q), ctypes.byref(r))
        return q.value, r.value

    def track_sums_of(self, lattice=None) -> np.ndarray:
        """Coordinate sums (Eq. 11) of a lattice (default: this state's) as
        tracking starts them, with this state's parameters: [n_cells + 1, 3]."""
        lat = self.lattice if lattice is None else np.ascontiguousarray(lattice, dtype=np.int32)
        V = np.zeros(self.w.n_cells + 1, dtype=np.int32)
        A = np.zeros_like(V)
        lib().orc_recount(ctypes.byref(self.params), _ptr(lat, ctypes.c_int32), _ptr(V, ctypes.c_int32),
                          _ptr(A, ctypes.c_int32))
        S = np.zeros((self.w.n_cells + 1, 3), dtype=np.int64)
        lib().orc_track_init(ctypes.byref(self.params), _ptr(lat, ctypes.c_int32), _ptr(V, ctypes.c_int32),
                             _ptr(S, ctypes.c_int64))
        return S

    def centroids(self) -> np.ndarray:
        X = np.zeros((self.w.n_cells + 1, 3))
        lib().orc_centroids(ctypes.byref(self.params), _ptr(self.lattice, ctypes.c_int32), _ptr(X, ctypes.c_double))
        return X

    def recount(self):
        V = np.zeros_like(self.V)
        A = np.zeros_like(self.A)
        lib().orc_recount(ctypes.byref(self.params), _ptr(self.lattice, ctypes.c_int32),
                          _ptr(V, ctypes.c_int32), _ptr(A, ctypes.c_int32))
        return V, A

    def delta_h(self, j: int, n_idx: int):
        """All energy terms of one attempt (target j, source = neighbour n_idx)."""
        r = [ctypes.c_int64(0), ctypes.c_int64(0), ctypes.c_double(0), ctypes.c_int64(0),
             ctypes.c_int64(0), ctypes.c_double(0), ctypes.c_double(0)]
        rc = lib().orc_delta_h(ctypes.byref(self.params), _ptr(self.lattice, ctypes.c_int32),
                               _ptr(self.act, ctypes.c_uint8), _ptr(self.V, ctypes.c_int32),
                               _ptr(self.A, ctypes.c_int32), j, n_idx, *[ctypes.byref(x) for x in r])
        if rc != 0:
            raise RuntimeError("orc_delta_h failed")
        keys = ["dh_int", "dh_act_q", "dh_act_real", "gm_i_q", "gm_j_q", "gm_i", "gm_j"]
        return {k: x.value for k, x in zip(keys, r)}


def make_params(w, cell_type: np.ndarray, state=None) -> Params:
    p = Params()
    p.dim, p.nx, p.ny, p.nz = w.dim, w.nx, w.ny, w.nz
    for a in range(MAXT):
        for b in range(MAXT):
            p.J[a][b] = int(w.J[a, b])
        p.lambda_v[a] = int(w.lambda_v[a])
        p.v_target[a] = int(w.v_target[a])
        p.lambda_p[a] = int(w.lambda_p[a])
        p.a_target[a] = int(w.a_target[a])
        p.lambda_act[a] = int(w.lambda_act[a])
        p.max_act[a] = int(w.max_act[a])
    p.T = float(w.T)
    p.obstacle_type = w.obstacle_type
    p.a, p.c, p.P = w.a, w.c, w.P
    p.seed = w.seed
    p.n_cells = w.n_cells
    p.cell_type = cell_type.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8))
    p.tile = int(getattr(w, "tile", 0))
    p.tile_cycles = int(getattr(w, "tile_cycles", 1))
    if state is not None and state.chem is not None:
        p.chem_field = _ptr(state.chem, ctypes.c_int16)
    for name in ("lambda_chem", "lambda_pers", "dt_pers"):
        v = getattr(w, name, None)
        if v is not None:
            arr = getattr(p, name)
            for a in range(MAXT):
                arr[a] = int(v[a])
    if getattr(w, "mu_pers", None) is not None:
        for a in range(MAXT):
            p.mu_pers[a] = float(w.mu_pers[a])
    if state is not None and state.pers_dir is not None:
        p.pers_dir = _ptr(state.pers_dir, ctypes.c_double)
        p.pers_hist = _ptr(state.pers_hist, ctypes.c_double)
        p.pers_hist_len = state.pers_len
        p.pers_t0 = 0
    return p


def philox4x32_10(ctr, key):
    c = (ctypes.c_uint32 * 4)(*[int(x) & 0xFFFFFFFF for x in ctr])
    k = (ctypes.c_uint32 * 2)(*[int(x) & 0xFFFFFFFF for x in key])
    o = (ctypes.c_uint32 * 4)()
    lib().orc_philox4x32_10(c, k, o)
    return [int(x) for x in o]


def thr_table(T: float) -> np.ndarray:
    cap = int(16.0 * T * 32.0 * 0.6931471805599453) + 64
    buf = np.zeros(cap, dtype=np.uint32)
    L = lib().orc_thr_table(T, _ptr(buf, ctypes.c_uint32), cap)
    if L < 0:
        raise RuntimeError("threshold table did not reach zero")
    return buf[:L].copy()


def ln_table() -> np.ndarray:
    t = np.zeros(129, dtype=np.int32)
    lib().orc_ln_table(_ptr(t, ctypes.c_int32))
    return t


def expq_table() -> np.ndarray:
    n = lib().orc_expq_size()
    t = np.zeros(n, dtype=np.int32)
    lib().orc_expq_table(_ptr(t, ctypes.c_int32), n)
    return t


def colour_perm(w, t: int, pc: int) -> list:
    ct = np.ascontiguousarray(w.cell_type, dtype=np.uint8)
    p = make_params(w, ct)
    perm = (ctypes.c_int32 * 27)()
    C = lib().orc_colour_perm(ctypes.byref(p), t, pc, perm)
    return [int(perm[i]) for i in range(C)]


def subpass_targets(w, t: int, sp: int) -> np.ndarray:
    """Target site of every attempt of sub-pass sp of MCS t (oracle (b)'s
    schedule), in (block, round) order."""
    ct = np.ascontiguousarray(w.cell_type, dtype=np.uint8)
    p = make_params(w, ct)
    out = np.zeros(w.n_sites, dtype=np.int64)
    n = lib().orc_subpass_targets(ctypes.byref(p), t, sp, _ptr(out, ctypes.c_int64))
    return out[:n].copy()


def tile_offset(w, t: int) -> np.ndarray:
    """Offset (x, y, z) of the tile grid of the tiled schedule in MCS t."""
    ct = np.ascontiguousarray(w.cell_type, dtype=np.uint8)
    p = make_params(w, ct)
    off = np.zeros(3, dtype=np.int64)
    lib().orc_tile_offset_of(ctypes.byref(p), t, _ptr(off, ctypes.c_int64))
    return off


def neighbour_offsets(dim: int) -> np.ndarray:
    off = np.zeros((26, 3), dtype=np.int32)
    n = lib().orc_neighbour_offsets(dim, _ptr(off, ctypes.c_int32))
    return off[:n].copy()
