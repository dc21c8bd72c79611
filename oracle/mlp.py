"""FP64 CPU oracle for the MLP-ensemble emulator: test infrastructure only.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU legs may
import this module.  It shares no code with the CUDA kernels.

The emulator maps the seven swept CPM parameters (J cell-cell, J
cell-medium, lambda_V, lambda_P, lambda_Act, Max_Act, T) to sixteen summary
statistics of a run.  Each member of the ensemble is a fully connected
network

    Z_l = H_{l-1} W_l^T + b_l,   H_l = GELU(Z_l)   (hidden layers l = 1..L-1)
    P   = H_{L-1} W_L^T + b_L                       (linear output layer)

with GELU(z) = z Phi(z), Phi the standard normal CDF (Hendrycks & Gimpel
2016), trained on the mean squared error

    loss = (1 / (n_rows n_out)) sum (P - Y)^2

with Adam (Kingma & Ba 2015, Algorithm 1):

    m <- b1 m + (1 - b1) g,   v <- b2 v + (1 - b2) g^2,
    w <- w - lr (m / (1 - b1^t)) / (sqrt(v / (1 - b2^t)) + eps).

Everything here is float64.  The backward pass is the chain rule written out
layer by layer (dP = 2 (P - Y) / (n_rows n_out); dW_l = dZ_l^T H_{l-1};
db_l = column sums of dZ_l; dH_{l-1} = dZ_l W_l; dZ_l = dH_l GELU'(Z_l) with
GELU'(z) = Phi(z) + z phi(z)).

Parameters of one member are a list of (W [out, in], b [out]) pairs.
"""
from __future__ import annotations

import math

import numpy as np

try:
    from scipy.special import erf as _erf
except ImportError:  # pragma: no cover - scipy is in both images
    _erf = np.vectorize(math.erf)

SQRT2 = math.sqrt(2.0)
INV_SQRT_2PI = 1.0 / math.sqrt(2.0 * math.pi)


def gelu(z):
    z = np.asarray(z, dtype=np.float64)
    return 0.5 * z * (1.0 + _erf(z / SQRT2))


def gelu_grad(z):
    z = np.asarray(z, dtype=np.float64)
    return 0.5 * (1.0 + _erf(z / SQRT2)) + z * INV_SQRT_2PI * np.exp(-0.5 * z * z)


def forward(params, X):
    """One member: returns (P, cache) with cache = (inputs H_{l-1}, pre-activations Z_l)."""
    H = np.asarray(X, dtype=np.float64)
    Hs, Zs = [], []
    for l, (W, b) in enumerate(params):
        Hs.append(H)
        Z = H @ np.asarray(W, np.float64).T + np.asarray(b, np.float64)
        Zs.append(Z)
        H = Z if l == len(params) - 1 else gelu(Z)
    return H, (Hs, Zs)


def mse(P, Y):
    """Mean squared error over all elements and its gradient with respect to P."""
    P = np.asarray(P, np.float64)
    D = P - np.asarray(Y, np.float64)
    n = D.size
    return float((D * D).sum() / n), 2.0 * D / n


def backward(params, cache, dP):
    """Gradients [(dW_l, db_l)] of the loss whose gradient with respect to
    the output is dP."""
    Hs, Zs = cache
    grads = [None] * len(params)
    dZ = np.asarray(dP, np.float64)
    for l in range(len(params) - 1, -1, -1):
        W = np.asarray(params[l][0], np.float64)
        grads[l] = (dZ.T @ Hs[l], dZ.sum(axis=0))
        if l > 0:
            dH = dZ @ W
            dZ = dH * gelu_grad(Zs[l - 1])
    return grads


def loss_and_grads(params, X, Y):
    P, cache = forward(params, X)
    loss, dP = mse(P, Y)
    return loss, backward(params, cache, dP), P


def adam(w, g, m, v, lr, b1, b2, eps, t):
    """One Adam update of step t >= 1 (Kingma & Ba 2015, Algorithm 1);
    returns new (w, m, v)."""
    w = np.asarray(w, np.float64)
    m = b1 * np.asarray(m, np.float64) + (1.0 - b1) * g
    v = b2 * np.asarray(v, np.float64) + (1.0 - b2) * g * g
    mhat = m / (1.0 - b1 ** t)
    vhat = v / (1.0 - b2 ** t)
    return w - lr * mhat / (np.sqrt(vhat) + eps), m, v


def ensemble_predict(members, X):
    """Mean and (population) standard deviation over the members' outputs."""
    outs = np.stack([forward(p, X)[0] for p in members])
    return outs.mean(axis=0), outs.std(axis=0), outs


def fallback_mask(std, rmse, factor=3.0):
    """A query point falls back to the CPM when, for any statistic, the
    ensemble's standard deviation exceeds factor x that statistic's
    validation RMSE (both in the standardised units the network predicts)."""
    return (np.asarray(std) > factor * np.asarray(rmse)[None, :]).any(axis=1)
