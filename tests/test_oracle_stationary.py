"""Oracle (a) against the exactly solved Markov chain of a tiny CPM.

A 4x4 periodic Moore-8 lattice holds two cells and no medium, so a state is a
16-bit pattern (which sites belong to cell 1); the two patterns in which a
cell has vanished are excluded, as the chain forbids them.  From every state
the transition matrix of the serial CPM (Methods, Eq. 1 to Eq. 3: target j
uniform, source i uniform among j's 8 neighbours, acceptance min(1,
exp(-dH/T))) is built with dH taken as a brute-force difference of the full
Hamiltonian; the stationary distribution pi solves pi P = pi.  The CPM
proposal is not symmetric, so pi is not the Boltzmann distribution: the test
needs the exact matrix.  The serial oracle's long-run histogram of the volume
and perimeter of cell 1 must agree with pi within batch-means error.
"""
import numpy as np
import pytest
import scipy.sparse as sp

import cpm_workloads as cw
import oracle
from tests import brute

L = 4
NS = L * L


def _workload(T, lam_v, v_t, lam_p, a_t, j11):
    w = cw.random_small(1, dim=2, n=L, n_cells=2, edge=1, perimeter=True, a=4)
    w.J[:] = 0
    w.J[1, 1] = j11
    w.lambda_v[:] = 0
    w.lambda_p[:] = 0
    w.lambda_v[1] = lam_v
    w.v_target[1] = v_t
    w.lambda_p[1] = lam_p
    w.a_target[1] = a_t
    w.cell_type = np.array([0, 1, 1], dtype=np.uint8)
    return w.replace(T=float(T))


def _all_states():
    s = np.arange(1 << NS, dtype=np.int64)
    bits = (s[:, None] >> np.arange(NS)[None, :]) & 1
    lat = np.where(bits == 1, 1, 2).astype(np.int32).reshape(-1, 1, L, L)
    return s, lat


def _energies(w, lat):
    H = brute.hamiltonian_batch(w, lat).astype(np.float64)
    V1 = (lat == 1).reshape(len(lat), -1).sum(1)
    A1 = np.zeros(len(lat), dtype=np.int64)
    for o in brute.offsets(2):
        nb = np.roll(lat, shift=tuple(-x for x in o), axis=(1, 2, 3))
        A1 += ((lat == 1) & (nb != 1)).reshape(len(lat), -1).sum(1)
    # spot-check the batched forms against the single-lattice definitions
    for k in (1, 77, 4097, 40000):
        assert H[k] == brute.hamiltonian(w, lat[k])
        assert A1[k] == brute.interfaces(w, lat[k])[1]
    return H, V1, A1


def _exact_pi(w):
    s, lat = _all_states()
    H, V1, A1 = _energies(w, lat)
    off = brute.offsets(2)
    valid = (s != 0) & (s != (1 << NS) - 1)
    rows, cols, vals = [], [], []
    stay = np.zeros(len(s))
    for j in range(NS):
        jy, jx = divmod(j, L)
        for (_, dy, dx) in off:
            i = ((jy + dy) % L) * L + (jx + dx) % L
            bj = (s >> j) & 1
            bi = (s >> i) & 1
            move = valid & (bj != bi)
            # target cell loses its last site? (cell 1 has V1 sites, cell 2 has NS-V1)
            vj = np.where(bj == 1, V1, NS - V1)
            move &= vj > 1
            t = s ^ (1 << j)
            dH = H[t] - H[s]
            p = np.where(move, np.minimum(1.0, np.exp(-dH / w.T)), 0.0) / (NS * 8)
            rows.append(s[move])
            cols.append(t[move])
            vals.append(p[move])
            stay += p
    rows = np.concatenate(rows)
    cols = np.concatenate(cols)
    vals = np.concatenate(vals)
    n = len(s)
    P = sp.csr_matrix((vals, (rows, cols)), shape=(n, n))
    P = P + sp.diags(np.where(valid, 1.0 - stay, 0.0))
    pi = np.where(valid, 1.0, 0.0)
    pi /= pi.sum()
    PT = P.T.tocsr()
    for it in range(20000):
        new = PT @ pi
        if np.abs(new - pi).sum() < 1e-13:
            pi = new
            break
        pi = new
    pi /= pi.sum()
    return pi, V1, A1


@pytest.mark.parametrize("params", [
    dict(T=6.0, lam_v=1, v_t=8, lam_p=0, a_t=0, j11=4),
    dict(T=10.0, lam_v=2, v_t=6, lam_p=1, a_t=20, j11=6),
])
def test_serial_chain_matches_exact_stationary_distribution(params):
    w = _workload(**params)
    pi, V1, A1 = _exact_pi(w)
    # exact marginals of (V1) and of (A1)
    pv = np.bincount(V1, weights=pi, minlength=NS + 1)
    amax = int(A1.max()) + 1
    pa = np.bincount(A1, weights=pi, minlength=amax)

    # long serial run, one sample per MCS, batch means for the error bars
    st = oracle.State(w.replace(seed=12345))
    st.lattice[:] = np.where(np.arange(NS).reshape(1, L, L) < NS // 2, 1, 2)
    st.V[:], st.A[:] = st.recount()
    st.serial_run(200)  # burn-in
    n_batches, per_batch = 20, 4000
    hv = np.zeros((n_batches, NS + 1))
    ha = np.zeros((n_batches, amax))
    for b in range(n_batches):
        for _ in range(per_batch):
            st.serial_run(1)
            hv[b, st.V[1]] += 1
            ha[b, st.A[1]] += 1
    hv /= per_batch
    ha /= per_batch
    for emp, exact in ((hv, pv), (ha, pa)):
        m = emp.mean(0)
        se = emp.std(0, ddof=1) / np.sqrt(n_batches)
        z = np.abs(m - exact[: len(m)]) / np.maximum(se, 2e-4)
        assert np.all(z < 5.0), (m, exact, z)
        assert 0.5 * np.abs(m - exact[: len(m)]).sum() < 0.02
