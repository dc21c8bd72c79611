"""Statistics of the 3D Act tissue for the parallel-versus-serial comparison
(the paper validates its scheme by the behaviour of the simulated cells:
Results, "Aligning the lattice update statistics", Fig. 3-5).

Shared by the GPU test and by the script that stores the serial chain's
statistics (tests/golden/make_tissue_serial_stats.py), so both sides reduce
their runs identically.  Analysis only: no CPM arithmetic lives here.

Protocol: the 3D fibre tissue (Act on, perimeter, obstacles) at 128^3,
BURN MCS from the seed cubes (cells reach V_t within about 20 MCS and the
acceptance rate settles by about 100), then SNAPS snapshots EVERY MCS apart.
Per run: cell volume mean and variance and interface-count mean (over live
cells and snapshots), acceptance rate over the window, and the mean squared
displacement of cell centroids over 10 and 50 MCS (all windows of that lag
inside the observation window).
"""
import numpy as np

N = 128
BURN, SNAPS, EVERY = 100, 40, 10
STATS = ("vmean", "vvar", "amean", "acc", "msd10", "msd50")


def centroids(lat, n_cells: int):
    """Periodic centroid of every cell id 0..n_cells (circular mean along
    each axis) of a (nz, ny, nx) int32 lattice (torch tensor on any device,
    or numpy array), float64 [n_cells + 1, 3] of the same kind."""
    if isinstance(lat, np.ndarray):
        return _centroids_np(lat, n_cells)
    import torch
    ids = lat.reshape(-1).long()
    m = ids > 0
    idx = torch.nonzero(m).squeeze(1)
    ids = ids[idx]
    out = torch.zeros((n_cells + 1, 3), dtype=torch.float64, device=lat.device)
    stride = 1
    dims = list(lat.shape)
    for axis in (2, 1, 0):
        L = dims[axis]
        coord = (idx // stride) % L
        stride *= L
        ang = coord.double() * (2 * np.pi / L)
        cs = torch.bincount(ids, weights=torch.cos(ang), minlength=n_cells + 1)
        sn = torch.bincount(ids, weights=torch.sin(ang), minlength=n_cells + 1)
        out[:, axis] = torch.remainder(torch.atan2(sn, cs), 2 * np.pi) * (L / (2 * np.pi))
    return out


def _centroids_np(lat: np.ndarray, n_cells: int) -> np.ndarray:
    ids = lat.reshape(-1).astype(np.int64)
    idx = np.nonzero(ids > 0)[0]
    ids = ids[idx]
    out = np.zeros((n_cells + 1, 3))
    stride = 1
    for axis in (2, 1, 0):
        L = lat.shape[axis]
        coord = (idx // stride) % L
        stride *= L
        ang = coord * (2 * np.pi / L)
        cs = np.bincount(ids, weights=np.cos(ang), minlength=n_cells + 1)
        sn = np.bincount(ids, weights=np.sin(ang), minlength=n_cells + 1)
        out[:, axis] = np.remainder(np.arctan2(sn, cs), 2 * np.pi) * (L / (2 * np.pi))
    return out


class Recorder:
    """Accumulates one run's snapshots: centroids (unwrapped across
    snapshots by the minimal image), tallies and the accepted-copy count."""

    def __init__(self, shape, n_cells: int):
        self.L = np.array(shape, dtype=np.float64)
        self.n_cells = n_cells
        self.traj, self.prev = [], None
        self.V, self.A = [], []

    def snapshot(self, lat, V=None, A=None):
        c = centroids(lat, self.n_cells)
        if not isinstance(c, np.ndarray):
            c = c.cpu().numpy()
        if self.prev is None:
            self.traj.append(np.zeros_like(c))
        else:
            d = c - self.prev
            d -= np.round(d / self.L) * self.L
            self.traj.append(self.traj[-1] + d)
        self.prev = c
        if V is not None:
            self.V.append(np.asarray(V, dtype=np.float64)[1:])
            self.A.append(np.asarray(A, dtype=np.float64)[1:])

    def summary(self, accepts: int, n_sites: int) -> dict:
        traj = np.stack(self.traj)[:, 1:, :]
        V, A = np.array(self.V), np.array(self.A)
        live = V > 0
        lag = lambda k: float(((traj[k:] - traj[:-k]) ** 2).sum(-1).mean())
        return dict(vmean=float(V[live].mean()), vvar=float(V[live].var()), amean=float(A[live].mean()),
                    acc=accepts / ((len(self.traj) - 1) * EVERY * n_sites),
                    msd10=lag(10 // EVERY), msd50=lag(50 // EVERY))
