"""MLP-ensemble emulator of CPM summary statistics (include/cpm_emulator.h).

The emulator maps the seven swept CPM parameters (J cell-cell, J
cell-medium, lambda_V, lambda_P, lambda_Act, Max_Act, T; the energy terms of
Methods Eq. 1, Eq. 3 and Eq. 8) to sixteen summary statistics of a run.  It
is trained on runs of the batched CPM (cpm_batch_*), its network is trained
and evaluated by the library's own kernels (cpm_mlp_*), and the CPM remains
both its judge and its fallback: a query whose ensemble disagreement exceeds
``factor`` x the validation RMSE of any statistic is simulated instead.

Pieces:
* ``Ensemble``       -- the network (cpm_mlp handle): gradients, Adam
  training, raw outputs, prediction with the fallback flag.
* ``simulate``       -- runs of the batched CPM observed every ``every`` MCS
  through cpm_batch_observe and reduced on the GPU by cpm_batch_summarize.
* ``Emulator``       -- target transform, 80/20 split, training, validation
  RMSE, prediction, and ``sweep`` (emulator + CPM fallback).

Everything that touches a lattice, an observation or a network runs in the
CUDA library; the host marshals arguments and applies the affine target
transform of the training set.
"""
from __future__ import annotations

import ctypes
import math
import time
import warnings

import numpy as np

from . import cpm

STATS = [
    "vol_mean",      # mean cell volume / V_t
    "vol_sd",        # standard deviation of cell volume over cells / V_t
    "perim_mean",    # mean interface count (Eq. 3) / A_t
    "perim_sd",      # standard deviation of the interface count over cells / A_t
    "msd10",         # mean squared centroid displacement over 10 MCS (sites^2)
    "msd50",         # ... over 50 MCS
    "msd200",        # ... over 200 MCS
    "speed_mean",    # mean centroid speed over 10-MCS steps (sites / MCS)
    "speed_sd",      # its standard deviation
    "dac50",         # directional autocorrelation of successive 50-MCS displacements (mean cosine)
    "persistence",   # integral of the step-direction autocorrelation up to its first zero (MCS)
    "arrest",        # fraction of 50-MCS sub-tracks slower than 0.05 sites / MCS
    "acceptance",    # accepted copies / copy attempts
    "contact_cc",    # cell-cell share of the cells' interface pairs
    "straightness",  # net displacement / path length over the window
    "elongation",    # sqrt of the ratio of the principal second moments of a cell
]
LOG_STATS = {"vol_sd", "perim_sd", "msd10", "msd50", "msd200", "speed_mean", "speed_sd", "persistence",
             "elongation"}


# --------------------------------------------------------------------------
# the network
# --------------------------------------------------------------------------

def _torch():
    import torch
    return torch


def _dptr(t):
    torch = _torch()
    assert isinstance(t, torch.Tensor) and t.is_cuda and t.is_contiguous()
    return ctypes.c_void_p(t.data_ptr())


class Ensemble:
    """n_members MLPs n_in -> width x n_hidden (GELU) -> n_out on the GPU."""

    def __init__(self, init_params, n_members=5, n_in=7, width=256, n_hidden=4, n_out=16, max_rows=8192,
                 stream=None):
        lib = cpm.load()
        self.lib = lib
        self.shape = cpm.MlpShape(n_members, n_in, width, n_hidden, n_out, max_rows)
        self.P = int(lib.cpm_mlp_param_count(ctypes.byref(self.shape)))
        if self.P < 0:
            raise ValueError("invalid network shape")
        init = np.ascontiguousarray(init_params, dtype=np.float32).reshape(n_members, self.P)
        h = ctypes.c_void_p()
        st = 0 if stream is None else int(getattr(stream, "cuda_stream", stream))
        rc = lib.cpm_mlp_create(ctypes.byref(self.shape), init.ctypes.data_as(ctypes.c_void_p), ctypes.c_void_p(st),
                                ctypes.byref(h))
        if rc != 0:
            raise cpm.CPMError(rc, "cpm_mlp_create: " + lib.cpm_mlp_last_error(None).decode())
        self.h = h
        self.sizes = [n_in] + [width] * n_hidden + [n_out]

    def _check(self, rc):
        if rc != 0:
            raise cpm.CPMError(rc, self.lib.cpm_mlp_last_error(self.h).decode())

    @property
    def n_members(self):
        return self.shape.n_members

    def get_params(self) -> np.ndarray:
        out = np.empty((self.n_members, self.P), dtype=np.float32)
        self._check(self.lib.cpm_mlp_get_params(self.h, out.ctypes.data_as(ctypes.c_void_p)))
        return out

    def set_params(self, params):
        p = np.ascontiguousarray(params, dtype=np.float32).reshape(self.n_members, self.P)
        self._check(self.lib.cpm_mlp_set_params(self.h, p.ctypes.data_as(ctypes.c_void_p)))

    def grads(self, X, Y, order=None, offset=0, rows=None):
        """Gradients [n_members, P] and losses [n_members] of one batch (device tensors in and out)."""
        torch = _torch()
        rows = X.shape[0] if rows is None else rows
        g = torch.empty((self.n_members, self.P), dtype=torch.float32, device=X.device)
        loss = torch.empty(self.n_members, dtype=torch.float32, device=X.device)
        self._check(self.lib.cpm_mlp_grads(self.h, _dptr(X), _dptr(Y), X.shape[0],
                                           _dptr(order) if order is not None else None, offset, rows, _dptr(g),
                                           _dptr(loss)))
        return g, loss

    def train(self, X, Y, order, batch_rows, lr, beta1=0.9, beta2=0.999, eps=1e-8, trace=False):
        """Adam steps over consecutive batches of ``order`` (int32 device tensor)."""
        torch = _torch()
        steps = order.shape[0] // batch_rows
        lt = torch.empty((max(steps, 1), self.n_members), dtype=torch.float32, device=X.device) if trace else None
        self._check(self.lib.cpm_mlp_train(self.h, _dptr(X), _dptr(Y), X.shape[0], _dptr(order), order.shape[0],
                                           batch_rows, lr, beta1, beta2, eps, _dptr(lt) if trace else None))
        return lt[:steps] if trace else None

    def forward(self, X):
        torch = _torch()
        out = torch.empty((self.n_members, X.shape[0], self.shape.n_out), dtype=torch.float32, device=X.device)
        self._check(self.lib.cpm_mlp_forward(self.h, _dptr(X), X.shape[0], _dptr(out)))
        return out

    def set_output_transform(self, shift, scale, log_mask, val_rmse=None, factor=3.0):
        f = lambda a: np.ascontiguousarray(a, dtype=np.float32)  # noqa: E731
        sh, sc = f(shift), f(scale)
        lm = np.ascontiguousarray(log_mask, dtype=np.uint8)
        rm = f(val_rmse) if val_rmse is not None else None
        self._keep = (sh, sc, lm, rm)
        self._check(self.lib.cpm_mlp_set_output_transform(
            self.h, sh.ctypes.data_as(ctypes.c_void_p), sc.ctypes.data_as(ctypes.c_void_p),
            lm.ctypes.data_as(ctypes.c_void_p), rm.ctypes.data_as(ctypes.c_void_p) if rm is not None else None,
            float(factor)))

    def predict(self, X):
        """(mean [n, n_out] in the statistics' units, std [n, n_out] standardised, fallback [n] uint8)."""
        torch = _torch()
        n = X.shape[0]
        mean = torch.empty((n, self.shape.n_out), dtype=torch.float32, device=X.device)
        std = torch.empty_like(mean)
        fb = torch.empty(n, dtype=torch.uint8, device=X.device)
        self._check(self.lib.cpm_mlp_predict(self.h, _dptr(X), n, _dptr(mean), _dptr(std), _dptr(fb)))
        return mean, std, fb

    def launches(self) -> int:
        return int(self.lib.cpm_mlp_kernel_launches(self.h))

    def close(self):
        if getattr(self, "h", None) is not None and self.h.value:
            self.lib.cpm_mlp_destroy(self.h)
            self.h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# --------------------------------------------------------------------------
# statistics of CPM runs
# --------------------------------------------------------------------------

def simulate(thetas, seeds, burn=200, window=800, every=10, chunk=2048, stream=None, timings=None):
    """Statistics [n, 16] (STATS order) of CPM runs at parameter points
    thetas [n, 7] (model units), one run per row with the given seeds, on
    the batched CPM: ``burn`` MCS, then ``window`` MCS observed every
    ``every`` MCS.  ``timings`` (dict, optional) accumulates seconds spent
    creating batches, simulating (observations and statistics included) and
    releasing them."""
    import cpm_workloads as cw
    torch = _torch()
    thetas = np.asarray(thetas, dtype=np.float64)
    seeds = np.asarray(seeds, dtype=np.int64)
    n = len(thetas)
    out = np.empty((n, len(STATS)))
    S = window // every
    tm = timings if timings is not None else {}
    for c0 in range(0, n, chunk):
        t0 = time.perf_counter()
        ws = [cw.emulator_run(thetas[i], int(seeds[i])) for i in range(c0, min(n, c0 + chunk))]
        b = cpm.Batch(ws, stream=stream)
        t1 = time.perf_counter()
        rows = int(b.observation_rows()[-1])
        cells = torch.empty((S + 1, rows, cpm.OBS_FIELDS), dtype=torch.int64, device="cuda")
        member = torch.empty((S + 1, len(ws), 2), dtype=torch.int64, device="cuda")
        b.step(burn)
        for s in range(S + 1):
            b.observe(cells[s], member[s])
            if s < S:
                b.step(every)
        st = torch.empty((len(ws), len(STATS)), dtype=torch.float64, device="cuda")
        b.summarize(cells, member, every, st)
        out[c0:c0 + len(ws)] = st.cpu().numpy()
        t2 = time.perf_counter()
        tm["launches"] = tm.get("launches", 0) + b.launches()
        b.close()
        t3 = time.perf_counter()
        tm["create"] = tm.get("create", 0.0) + (t1 - t0)
        tm["cpm"] = tm.get("cpm", 0.0) + (t2 - t1)
        tm["close"] = tm.get("close", 0.0) + (t3 - t2)
        tm["attempts"] = tm.get("attempts", 0) + sum(w.nx * w.ny for w in ws) * (burn + window)
    return out


# --------------------------------------------------------------------------
# emulator
# --------------------------------------------------------------------------

class Emulator:
    """Fits an Ensemble to (parameter point, statistics) pairs and answers
    queries, with the CPM fallback rule."""

    def __init__(self, init_seed=1, n_members=5, width=256, n_hidden=4, max_rows=8192, factor=3.0, stream=None):
        import cpm_workloads as cw
        self.sizes = [7] + [width] * n_hidden + [len(STATS)]
        self.net = Ensemble(cw.mlp_init(init_seed, n_members, self.sizes), n_members, 7, width, n_hidden,
                            len(STATS), max_rows, stream)
        self.factor = factor
        self.log_mask = np.array([s in LOG_STATS for s in STATS], dtype=np.uint8)

    # input / target transforms
    def _x(self, thetas):
        return ((np.asarray(thetas, np.float64) - self.x_lo) / (self.x_hi - self.x_lo)).astype(np.float32)

    def _t(self, Y):
        Y = np.asarray(Y, np.float64)
        return np.where(self.log_mask[None, :] == 1, np.log(np.maximum(Y, 1e-6)), Y)

    def fit(self, thetas, Y, epochs=120, batch_rows=1024, lr=2e-3, lr_min=None, val_frac=0.2, seed=0,
            eval_every=10):
        """Train on rows with finite statistics; the last ``val_frac`` of a
        seeded permutation is the validation split.  The learning rate
        follows a cosine from ``lr`` to ``lr_min`` (default lr / 40); every
        ``eval_every`` epochs the validation RMSE of the ensemble mean is
        measured and the best parameters so far are kept (early stopping).
        Returns a history dict."""
        torch = _torch()
        lr_min = lr / 40.0 if lr_min is None else lr_min
        thetas = np.asarray(thetas, np.float64)
        Y = np.asarray(Y, np.float64)
        ok = np.isfinite(Y).all(axis=1)
        thetas, Y = thetas[ok], Y[ok]
        perm = np.random.default_rng(seed).permutation(len(Y))
        n_val = int(round(val_frac * len(Y)))
        tr, va = perm[: len(Y) - n_val], perm[len(Y) - n_val:]
        self.x_lo, self.x_hi = thetas[tr].min(axis=0), thetas[tr].max(axis=0)
        self.x_hi = np.where(self.x_hi > self.x_lo, self.x_hi, self.x_lo + 1.0)
        T = self._t(Y)
        self.mu = T[tr].mean(axis=0)
        self.sd = np.maximum(T[tr].std(axis=0), 1e-6)
        Z = ((T - self.mu) / self.sd).astype(np.float32)
        X = self._x(thetas)
        Xtr = torch.from_numpy(X[tr]).cuda()
        Ztr = torch.from_numpy(Z[tr]).cuda()
        Xva = torch.from_numpy(X[va]).cuda()
        g = torch.Generator(device="cuda")
        g.manual_seed(seed)
        hist = {"val": [], "n_train": len(tr), "n_val": n_val, "epochs": epochs}

        def val_rmse():
            out = self.net.forward(Xva).cpu().numpy()
            return np.sqrt(((out.mean(axis=0) - Z[va]) ** 2).mean(axis=0))

        best, best_params, best_ep = None, None, -1
        t0 = time.perf_counter()
        for ep in range(epochs):
            lr_ep = lr_min + 0.5 * (lr - lr_min) * (1 + math.cos(math.pi * ep / max(1, epochs)))
            order = torch.randperm(len(tr), generator=g, device="cuda").to(torch.int32)
            self.net.train(Xtr, Ztr, order, batch_rows, lr_ep)
            if n_val and ((ep + 1) % eval_every == 0 or ep == epochs - 1):
                r = val_rmse()
                hist["val"].append((ep + 1, float(r.mean())))
                if best is None or r.mean() < best.mean():
                    best, best_params, best_ep = r, self.net.get_params(), ep + 1
        torch.cuda.synchronize()
        hist["train_s"] = time.perf_counter() - t0
        if best_params is not None and best_ep != epochs:
            self.net.set_params(best_params)
        self.val_rmse = best if best is not None else np.ones(len(STATS))
        hist["val_rmse"] = self.val_rmse
        hist["best_epoch"] = best_ep
        self.val_idx = np.nonzero(ok)[0][va]
        self.net.set_output_transform(self.mu, self.sd, self.log_mask, self.val_rmse, self.factor)
        return hist

    def predict(self, thetas):
        """(statistics [n, 16], ensemble std [n, 16] standardised, fallback [n] bool) as numpy."""
        torch = _torch()
        X = torch.from_numpy(self._x(thetas)).cuda()
        m, s, f = self.net.predict(X)
        return m.cpu().numpy(), s.cpu().numpy(), f.cpu().numpy().astype(bool)

    def sweep(self, thetas, seed=0, replicates=1, timings=None, **sim):
        """Statistics at every point: the emulator's answer where the ensemble
        agrees, the mean of ``replicates`` CPM runs where it falls back."""
        Yhat, _, fb = self.predict(thetas)
        idx = np.nonzero(fb)[0]
        if idx.size:
            rep_th = np.repeat(np.asarray(thetas)[idx], replicates, axis=0)
            rep_seed = seed * 1000003 + np.arange(rep_th.shape[0])
            Ys = simulate(rep_th, rep_seed, timings=timings, **sim).reshape(idx.size, replicates, -1)
            with warnings.catch_warnings():
                warnings.simplefilter("ignore", RuntimeWarning)  # a statistic undefined in every replicate stays NaN
                Yhat[idx] = np.nanmean(Ys, axis=1)
        return Yhat, fb

    def close(self):
        self.net.close()
