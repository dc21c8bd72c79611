"""Python binding of the C ABI in include/cpm.h (libcpm_gb300.so).

Argument marshalling only: every step of the sweep runs in the library's CUDA
kernels.  Device buffers may be passed as torch CUDA tensors (their data
pointers are handed over), host buffers as numpy arrays.  The library must
have been built (``paper_2312_09317_gb300.build.build()``); importing this
module without it raises, so nothing silently falls back to another path.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

MAX_TYPES = 8

CPM_OK, CPM_E_INVALID, CPM_E_NOMEM, CPM_E_CUDA, CPM_E_HANDLE, CPM_E_STATE, CPM_E_LIMIT = 0, -1, -2, -3, -4, -5, -6
OBS_FIELDS = 12  # per-cell fields of cpm_batch_observe


class Config(ctypes.Structure):
    _fields_ = [
        ("dim", ctypes.c_int32), ("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("nz", ctypes.c_int32),
        ("J", (ctypes.c_int32 * MAX_TYPES) * MAX_TYPES),
        ("lambda_v", ctypes.c_int32 * MAX_TYPES), ("v_target", ctypes.c_int32 * MAX_TYPES),
        ("lambda_p", ctypes.c_int32 * MAX_TYPES), ("a_target", ctypes.c_int32 * MAX_TYPES),
        ("lambda_act", ctypes.c_int32 * MAX_TYPES), ("max_act", ctypes.c_int32 * MAX_TYPES),
        ("temperature", ctypes.c_double),
        ("obstacle_type", ctypes.c_int32),
        ("a", ctypes.c_int32), ("c", ctypes.c_int32), ("P", ctypes.c_int32),
        ("seed", ctypes.c_uint64),
        ("n_cells", ctypes.c_int32),
        ("cell_type", ctypes.POINTER(ctypes.c_uint8)),
        ("init_lattice", ctypes.POINTER(ctypes.c_int32)),
        ("init_act", ctypes.POINTER(ctypes.c_uint8)),
        ("t0", ctypes.c_int64),
        ("tile", ctypes.c_int32),
        ("tile_cycles", ctypes.c_int32),
        ("chem_field", ctypes.POINTER(ctypes.c_int16)),
        ("lambda_chem", ctypes.c_int32 * MAX_TYPES),
        ("lambda_pers", ctypes.c_int32 * MAX_TYPES),
        ("mu_pers", ctypes.c_double * MAX_TYPES),
        ("dt_pers", ctypes.c_int32 * MAX_TYPES),
    ]


class Stats(ctypes.Structure):
    _fields_ = [
        ("mcs", ctypes.c_int64), ("subpass", ctypes.c_int32), ("n_live_cells", ctypes.c_int32),
        ("attempts", ctypes.c_int64), ("accepts", ctypes.c_int64),
        ("volume_mean", ctypes.c_double), ("volume_var", ctypes.c_double),
        ("perimeter_mean", ctypes.c_double), ("perimeter_var", ctypes.c_double),
    ]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


# Every function the header declares, with its ctypes signature.
_SIGNATURES = {
    "cpm_create": (ctypes.c_int, [ctypes.POINTER(Config), ctypes.c_void_p, ctypes.POINTER(ctypes.c_void_p)]),
    "cpm_step": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int64]),
    "cpm_step_subpasses": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int64]),
    "cpm_read_lattice": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int]),
    "cpm_read_tallies": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int]),
    "cpm_read_act": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int]),
    "cpm_load_lattice": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int]),
    "cpm_stats": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(Stats)]),
    "cpm_read_persistence": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
    "cpm_track_centroids": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32]),
    "cpm_batch_track_centroids": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32]),
    "cpm_batch_read_centroid_sums": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p, ctypes.c_int]),
    "cpm_read_centroid_sums": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int]),
    "cpm_verify": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_int64)]),
    "cpm_kernel_launches": (ctypes.c_int64, [ctypes.c_void_p]),
    "cpm_last_error": (ctypes.c_char_p, [ctypes.c_void_p]),
    "cpm_destroy": (None, [ctypes.c_void_p]),
    "cpm_batch_create": (ctypes.c_int, [ctypes.POINTER(Config), ctypes.c_int32, ctypes.c_void_p,
                                        ctypes.POINTER(ctypes.c_void_p)]),
    "cpm_batch_step": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int64]),
    "cpm_batch_size": (ctypes.c_int32, [ctypes.c_void_p]),
    "cpm_batch_autotune": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.POINTER(ctypes.c_int32)]),
    "cpm_batch_set_persistent": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64]),
    "cpm_batch_read_lattice": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p, ctypes.c_int]),
    "cpm_batch_load_lattice": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p, ctypes.c_int]),
    "cpm_batch_read_tallies": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p,
                                              ctypes.c_int]),
    "cpm_batch_read_act": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p, ctypes.c_int]),
    "cpm_batch_stats": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.POINTER(Stats)]),
    "cpm_batch_kernel_launches": (ctypes.c_int64, [ctypes.c_void_p]),
    "cpm_batch_last_error": (ctypes.c_char_p, [ctypes.c_void_p]),
    "cpm_batch_destroy": (None, [ctypes.c_void_p]),
    "cpm_batch_observe": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "cpm_batch_summarize": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32,
                                           ctypes.c_int32, ctypes.c_void_p]),
    "cpm_step_noalloc": (ctypes.c_int, [ctypes.POINTER(Config), ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                        ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_int64,
                                        ctypes.c_void_p, ctypes.POINTER(ctypes.c_int64)]),
}


class MlpShape(ctypes.Structure):
    """cpm_mlp_shape (include/cpm_emulator.h)."""
    _fields_ = [("n_members", ctypes.c_int32), ("n_in", ctypes.c_int32), ("width", ctypes.c_int32),
                ("n_hidden", ctypes.c_int32), ("n_out", ctypes.c_int32), ("max_rows", ctypes.c_int32)]


_VP, _I64, _I32, _F = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_float
_SIGNATURES.update({
    "cpm_mlp_param_count": (_I64, [ctypes.POINTER(MlpShape)]),
    "cpm_mlp_create": (ctypes.c_int, [ctypes.POINTER(MlpShape), _VP, _VP, ctypes.POINTER(_VP)]),
    "cpm_mlp_set_params": (ctypes.c_int, [_VP, _VP]),
    "cpm_mlp_get_params": (ctypes.c_int, [_VP, _VP]),
    "cpm_mlp_grads": (ctypes.c_int, [_VP, _VP, _VP, _I64, _VP, _I64, _I32, _VP, _VP]),
    "cpm_mlp_train": (ctypes.c_int, [_VP, _VP, _VP, _I64, _VP, _I64, _I32, _F, _F, _F, _F, _VP]),
    "cpm_mlp_forward": (ctypes.c_int, [_VP, _VP, _I64, _VP]),
    "cpm_mlp_set_output_transform": (ctypes.c_int, [_VP, _VP, _VP, _VP, _VP, _F]),
    "cpm_mlp_predict": (ctypes.c_int, [_VP, _VP, _I64, _VP, _VP, _VP]),
    "cpm_mlp_kernel_launches": (ctypes.c_uint64, [_VP]),
    "cpm_mlp_last_error": (ctypes.c_char_p, [_VP]),
    "cpm_mlp_destroy": (ctypes.c_int, [_VP]),
    "cpm_mlp_report_next_tc_timeout": (ctypes.c_int, [_VP]),
    "cpm_mlp_gemm": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                    _VP, _I64, _I64, _VP, _I64, _I64, _VP, _I64, _VP, ctypes.c_int, _I64, _I64,
                                    _VP, _I64, _I64, ctypes.c_int, _VP]),
})

_lib = None


def library_path() -> str:
    return _build.LIB


def load(path: str | None = None):
    """Load libcpm_gb300.so (raises OSError/RuntimeError when it is absent)."""
    global _lib
    if _lib is None:
        p = path or library_path()
        if not os.path.exists(p):
            raise RuntimeError("libcpm_gb300.so is not built (%s); run __graft_entry__.build()" % p)
        lib = ctypes.CDLL(p)
        for name, (res, args) in _SIGNATURES.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
    return _lib


class CPMError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("CPM error %d: %s" % (code, msg))
        self.code = code


def _ptr(x):
    """Data pointer and is-device flag of a numpy array or torch tensor."""
    if isinstance(x, np.ndarray):
        assert x.flags["C_CONTIGUOUS"]
        return x.ctypes.data, 0
    if hasattr(x, "data_ptr"):
        assert x.is_contiguous()
        return x.data_ptr(), 1 if x.is_cuda else 0
    raise TypeError("expected a numpy array or a torch tensor")


def make_config(w, keep: list) -> Config:
    """Config for a cpm_workloads.Workload; arrays it points to are appended
    to ``keep`` so they outlive the call."""
    c = Config()
    c.dim, c.nx, c.ny, c.nz = w.dim, w.nx, w.ny, w.nz
    for a in range(MAX_TYPES):
        for b in range(MAX_TYPES):
            c.J[a][b] = int(w.J[a, b])
        c.lambda_v[a] = int(w.lambda_v[a])
        c.v_target[a] = int(w.v_target[a])
        c.lambda_p[a] = int(w.lambda_p[a])
        c.a_target[a] = int(w.a_target[a])
        c.lambda_act[a] = int(w.lambda_act[a])
        c.max_act[a] = int(w.max_act[a])
    c.temperature = float(w.T)
    c.obstacle_type = int(w.obstacle_type)
    c.a, c.c, c.P = w.a, w.c, w.P
    c.seed = int(w.seed)
    c.n_cells = int(w.n_cells)
    ct = np.ascontiguousarray(w.cell_type, dtype=np.uint8)
    lat = np.ascontiguousarray(w.lattice, dtype=np.int32)
    keep += [ct, lat]
    c.cell_type = ct.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8))
    c.init_lattice = lat.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))
    if w.act is not None:
        act = np.ascontiguousarray(w.act, dtype=np.uint8)
        keep.append(act)
        c.init_act = act.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8))
    c.t0 = 0
    c.tile = int(getattr(w, "tile", 0))
    c.tile_cycles = int(getattr(w, "tile_cycles", 1))
    if getattr(w, "chem_field", None) is not None:
        f = np.ascontiguousarray(w.chem_field, dtype=np.int16)
        keep.append(f)
        c.chem_field = f.ctypes.data_as(ctypes.POINTER(ctypes.c_int16))
    for name in ("lambda_chem", "lambda_pers", "dt_pers"):
        v = getattr(w, name, None)
        if v is not None:
            arr = getattr(c, name)
            for a in range(MAX_TYPES):
                arr[a] = int(v[a])
    if getattr(w, "mu_pers", None) is not None:
        for a in range(MAX_TYPES):
            c.mu_pers[a] = float(w.mu_pers[a])
    return c


class Sim:
    """One CPM lattice on the GPU (a cpm_handle)."""

    def __init__(self, w, stream=None):
        lib = load()
        keep: list = []
        cfg = make_config(w, keep)
        self.w = w
        h = ctypes.c_void_p()
        st = 0 if stream is None else int(getattr(stream, "cuda_stream", stream))
        rc = lib.cpm_create(ctypes.byref(cfg), ctypes.c_void_p(st), ctypes.byref(h))
        if rc != CPM_OK:
            raise CPMError(rc, lib.cpm_last_error(None).decode())
        self.h = h
        self.lib = lib

    def _check(self, rc):
        if rc != CPM_OK:
            raise CPMError(rc, self.lib.cpm_last_error(self.h).decode())

    def step(self, n_mcs: int = 1):
        self._check(self.lib.cpm_step(self.h, n_mcs))

    def step_subpasses(self, n: int):
        self._check(self.lib.cpm_step_subpasses(self.h, n))

    def read_lattice(self, out=None):
        if out is None:
            out = np.empty((self.w.nz, self.w.ny, self.w.nx), dtype=np.int32)
        p, dev = _ptr(out)
        self._check(self.lib.cpm_read_lattice(self.h, ctypes.c_void_p(p), dev))
        return out

    def read_tallies(self):
        V = np.empty(self.w.n_cells + 1, dtype=np.int32)
        A = np.empty(self.w.n_cells + 1, dtype=np.int32)
        self._check(self.lib.cpm_read_tallies(self.h, ctypes.c_void_p(V.ctypes.data),
                                              ctypes.c_void_p(A.ctypes.data), 0))
        return V, A

    def read_act(self, out=None):
        if out is None:
            out = np.empty((self.w.nz, self.w.ny, self.w.nx), dtype=np.uint8)
        p, dev = _ptr(out)
        self._check(self.lib.cpm_read_act(self.h, ctypes.c_void_p(p), dev))
        return out

    def read_persistence(self):
        """Persistence directions p_hat, (n_cells + 1) x 3 float64."""
        out = np.zeros((self.w.n_cells + 1, 3))
        self._check(self.lib.cpm_read_persistence(self.h, ctypes.c_void_p(out.ctypes.data)))
        return out

    def track_centroids(self, on: bool = True):
        """Start (or stop) composite variable tracking (Eq. 11) of the cells'
        coordinate sums."""
        self._check(self.lib.cpm_track_centroids(self.h, 1 if on else 0))

    def read_centroid_sums(self):
        """Tracked coordinate sums, (n_cells + 1) x 3 int64; centroid = S / V."""
        out = np.zeros((self.w.n_cells + 1, 3), dtype=np.int64)
        self._check(self.lib.cpm_read_centroid_sums(self.h, ctypes.c_void_p(out.ctypes.data), 0))
        return out

    def load_lattice(self, src):
        p, dev = _ptr(src)
        self._check(self.lib.cpm_load_lattice(self.h, ctypes.c_void_p(p), dev))

    def stats(self) -> dict:
        s = Stats()
        self._check(self.lib.cpm_stats(self.h, ctypes.byref(s)))
        return s.as_dict()

    def verify(self) -> int:
        n = ctypes.c_int64(0)
        self._check(self.lib.cpm_verify(self.h, ctypes.byref(n)))
        return n.value

    def launches(self) -> int:
        return int(self.lib.cpm_kernel_launches(self.h))

    def close(self):
        if getattr(self, "h", None) is not None and self.h.value:
            self.lib.cpm_destroy(self.h)
            self.h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Batch:
    """An ensemble of independent lattices advanced together (a cpm_batch)."""

    def __init__(self, workloads, stream=None):
        lib = load()
        self.ws = list(workloads)
        keep: list = []
        arr = (Config * len(self.ws))()
        for k, w in enumerate(self.ws):
            arr[k] = make_config(w, keep)
        b = ctypes.c_void_p()
        st = 0 if stream is None else int(getattr(stream, "cuda_stream", stream))
        rc = lib.cpm_batch_create(arr, len(self.ws), ctypes.c_void_p(st), ctypes.byref(b))
        if rc != CPM_OK:
            raise CPMError(rc, lib.cpm_batch_last_error(None).decode())
        self.b = b
        self.lib = lib

    def _check(self, rc):
        if rc != CPM_OK:
            raise CPMError(rc, self.lib.cpm_batch_last_error(self.b).decode())

    def __len__(self):
        return int(self.lib.cpm_batch_size(self.b))

    def autotune(self, n_mcs_each: int = 2) -> int:
        """Time the candidate CTA shapes on this batch (it advances) and keep the fastest."""
        k = ctypes.c_int32(-1)
        self._check(self.lib.cpm_batch_autotune(self.b, n_mcs_each, ctypes.byref(k)))
        return k.value

    def step(self, n_mcs: int = 1):
        self._check(self.lib.cpm_batch_step(self.b, n_mcs))

    def set_persistent(self, on: bool = True, max_polls: int = -1):
        """Run each step as one persistent cooperative launch (cpm_batch_set_persistent)."""
        self._check(self.lib.cpm_batch_set_persistent(self.b, 1 if on else 0, max_polls))

    def read_lattice(self, idx: int, out=None):
        w = self.ws[idx]
        if out is None:
            out = np.empty((w.nz, w.ny, w.nx), dtype=np.int32)
        p, dev = _ptr(out)
        self._check(self.lib.cpm_batch_read_lattice(self.b, idx, ctypes.c_void_p(p), dev))
        return out

    def load_lattice(self, idx: int, src):
        p, dev = _ptr(src)
        self._check(self.lib.cpm_batch_load_lattice(self.b, idx, ctypes.c_void_p(p), dev))

    def track_centroids(self, on: bool = True):
        """Composite variable tracking (Eq. 11) in every lattice of the batch."""
        self._check(self.lib.cpm_batch_track_centroids(self.b, 1 if on else 0))

    def read_centroid_sums(self, idx: int):
        out = np.zeros((self.ws[idx].n_cells + 1, 3), dtype=np.int64)
        self._check(self.lib.cpm_batch_read_centroid_sums(self.b, idx, ctypes.c_void_p(out.ctypes.data), 0))
        return out

    def read_tallies(self, idx: int):
        w = self.ws[idx]
        V = np.empty(w.n_cells + 1, dtype=np.int32)
        A = np.empty(w.n_cells + 1, dtype=np.int32)
        self._check(self.lib.cpm_batch_read_tallies(self.b, idx, ctypes.c_void_p(V.ctypes.data),
                                                    ctypes.c_void_p(A.ctypes.data), 0))
        return V, A

    def read_act(self, idx: int):
        w = self.ws[idx]
        out = np.empty((w.nz, w.ny, w.nx), dtype=np.uint8)
        self._check(self.lib.cpm_batch_read_act(self.b, idx, ctypes.c_void_p(out.ctypes.data), 0))
        return out

    def stats(self, idx: int) -> dict:
        s = Stats()
        self._check(self.lib.cpm_batch_stats(self.b, idx, ctypes.byref(s)))
        return s.as_dict()

    def observation_rows(self) -> np.ndarray:
        """First observation row of every lattice (its medium row) and, last, the total."""
        return np.concatenate([[0], np.cumsum([w.n_cells + 1 for w in self.ws])]).astype(np.int64)

    def observe(self, cells_out, member_out):
        """cpm_batch_observe into device int64 tensors cells_out [rows, 12] and
        member_out [n, 2] (asynchronous on the batch's stream)."""
        pc, dc = _ptr(cells_out)
        pm, dm = _ptr(member_out)
        if not (dc and dm):
            raise ValueError("observe writes device buffers")
        self._check(self.lib.cpm_batch_observe(self.b, ctypes.c_void_p(pc), ctypes.c_void_p(pm)))

    def summarize(self, cells_hist, member_hist, every: int, out):
        """cpm_batch_summarize: device tensors cells_hist [S, rows, 12],
        member_hist [S, n, 2] -> out [n, 16] float64 (asynchronous)."""
        pc, dc = _ptr(cells_hist)
        pm, dm = _ptr(member_hist)
        po, do = _ptr(out)
        if not (dc and dm and do):
            raise ValueError("summarize works on device buffers")
        self._check(self.lib.cpm_batch_summarize(self.b, ctypes.c_void_p(pc), ctypes.c_void_p(pm),
                                                 int(cells_hist.shape[0]), every, ctypes.c_void_p(po)))

    def launches(self) -> int:
        return int(self.lib.cpm_batch_kernel_launches(self.b))

    def close(self):
        if getattr(self, "b", None) is not None and self.b.value:
            self.lib.cpm_batch_destroy(self.b)
            self.b = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
