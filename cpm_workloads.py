"""Seeded synthetic workloads for the cellular Potts model (CPM) sweep.

This module only produces inputs: an initial int32 cell-id lattice, the
per-cell type table and the integer-scaled model parameters.  It holds no
part of the CPM's arithmetic (no energies, no acceptance, no tallies), so the
CPU oracle and the CUDA path can both consume it without sharing any of the
method's code.

Conventions shared by every consumer (they are data conventions, not code):

* lattice layout: x fastest, then y, then z (``idx = x + nx*(y + ny*z)``);
  2D lattices have ``nz == 1``;
* cell id 0 is the medium (type 0); ids 1..n_cells are cells; a negative id
  (-1) is a frozen obstacle ("fibre") site whose type is ``obstacle_type``;
* energies are integers: every J and lambda of the paper's model (Methods,
  Eq. 1 and the perimeter term) is multiplied by an integer scale ``S`` so
  that all of them become integers, and the temperature T is multiplied by
  the same S;
* checkerboard parameters: ``a`` is the edge of one schedule area, ``c`` the
  number of checkerboard divisions per axis (so ``c**dim`` colours and active
  blocks of edge ``s = a // c``), ``P`` the number of colour cycles per MCS.

The paper's own tissues come from segmented microscopy, which is not
available; the generators below stand in for them with seeded shapes of the
same kind (point or cube cells at blue-noise centres; a Voronoi-edge fibre
network for the stromal obstacle).
"""
from __future__ import annotations

import dataclasses
from typing import Optional

import numpy as np

MAX_TYPES = 8


@dataclasses.dataclass
class Workload:
    name: str
    dim: int
    nx: int
    ny: int
    nz: int
    J: np.ndarray            # int32 [MAX_TYPES, MAX_TYPES], symmetric, scaled
    lambda_v: np.ndarray     # int32 [MAX_TYPES], scaled
    v_target: np.ndarray     # int32 [MAX_TYPES]
    lambda_p: np.ndarray     # int32 [MAX_TYPES], scaled
    a_target: np.ndarray     # int32 [MAX_TYPES]
    lambda_act: np.ndarray   # int32 [MAX_TYPES], scaled
    max_act: np.ndarray      # int32 [MAX_TYPES]
    T: float                 # temperature, scaled by the same S
    scale: int               # the integer energy scale S
    a: int
    c: int
    P: int
    seed: int
    obstacle_type: int
    lattice: np.ndarray      # int32 [nz, ny, nx] (x fastest)
    cell_type: np.ndarray    # uint8 [n_cells + 1]; entry 0 is the medium
    act: Optional[np.ndarray] = None  # uint8 [nz, ny, nx] initial Act values
    n_mcs: int = 1
    tile: int = 0            # tiled schedule: tile edge T (0: global rounds)
    tile_cycles: int = 1     # tiled schedule: tile cycles per MCS
    # motility terms (Eq. 4 to Eq. 7); None = off
    chem_field: Optional[np.ndarray] = None   # int16 [nz, ny, nx, dim]: the field C in Q14 (16384 = 1)
    lambda_chem: Optional[np.ndarray] = None  # int32 [MAX_TYPES], scaled
    lambda_pers: Optional[np.ndarray] = None  # int32 [MAX_TYPES], scaled
    mu_pers: Optional[np.ndarray] = None      # float64 [MAX_TYPES]: persistence strength mu
    dt_pers: Optional[np.ndarray] = None      # int32 [MAX_TYPES]: look-back of the update, MCS

    @property
    def n_cells(self) -> int:
        return int(self.cell_type.shape[0] - 1)

    @property
    def n_sites(self) -> int:
        return self.nx * self.ny * self.nz

    @property
    def act_on(self) -> bool:
        return bool(np.any(self.lambda_act != 0))

    @property
    def pers_on(self) -> bool:
        return self.lambda_pers is not None and bool(np.any(self.lambda_pers != 0))

    @property
    def chem_on(self) -> bool:
        return self.chem_field is not None and self.lambda_chem is not None and bool(np.any(self.lambda_chem != 0))

    def replace(self, **kw) -> "Workload":
        return dataclasses.replace(self, **kw)


def _params(n_types: int = 3):
    z = lambda: np.zeros(MAX_TYPES, dtype=np.int32)  # noqa: E731
    return (np.zeros((MAX_TYPES, MAX_TYPES), dtype=np.int32), z(), z(), z(), z(), z(), z())


def _sym(J, a, b, v):
    J[a, b] = v
    J[b, a] = v


# --------------------------------------------------------------------------
# seeding helpers
# --------------------------------------------------------------------------

def jittered_centres(shape, spacing: float, jitter: float, rng) -> np.ndarray:
    """Blue-noise centres: one point per cell of a regular grid of the given
    spacing, displaced uniformly by at most ``jitter`` per axis.  Any two
    centres are at least ``spacing - 2*jitter`` apart along some axis."""
    axes = []
    for n in shape:
        m = max(1, int(round(n / spacing)))
        axes.append((np.arange(m) + 0.5) * (n / m))
    grid = np.stack(np.meshgrid(*axes, indexing="ij"), axis=-1).reshape(-1, len(shape))
    grid = grid + rng.uniform(-jitter, jitter, size=grid.shape)
    pts = np.floor(grid).astype(np.int64)
    for d, n in enumerate(shape):
        pts[:, d] %= n
    return pts


def place_cubes(lattice: np.ndarray, centres: np.ndarray, edge: int) -> int:
    """Write cubes (squares in 2D) of the given edge, periodic, with ids
    1..len(centres) in centre order.  A site claimed by several cubes goes to
    the lowest id; sites that are not medium (obstacles) are left alone.
    Returns the number of cells (len(centres))."""
    dim = lattice.ndim
    shape = np.array(lattice.shape, dtype=np.int64)
    lo = -(edge // 2)
    offs = np.stack(np.meshgrid(*([np.arange(lo, lo + edge)] * dim), indexing="ij"),
                    axis=-1).reshape(-1, dim)
    n = len(centres)
    if n == 0:
        return 0
    flat = np.zeros(n * len(offs), dtype=np.int64)
    stride = 1
    for d in reversed(range(dim)):
        coord = (centres[:, None, d].astype(np.int64) + offs[None, :, d]) % shape[d]
        flat += coord.reshape(-1) * stride
        stride *= shape[d]
    ids = np.repeat(np.arange(1, n + 1, dtype=np.int32), len(offs))
    # first claim (lowest id) per site
    order = np.argsort(flat, kind="stable")
    fs = flat[order]
    first = np.ones(len(fs), dtype=bool)
    first[1:] = fs[1:] != fs[:-1]
    sites = fs[first]
    owner = ids[order][first]
    lv = lattice.reshape(-1)
    free = lv[sites] == 0
    lv[sites[free]] = owner[free]
    return n


# --------------------------------------------------------------------------
# the workloads
# --------------------------------------------------------------------------

def point_cells_2d(seed: int = 1, n: int = 200, n_cells: int = 100, a: int = 4, c: int = 2,
               P: int = 1, n_mcs: int = 500) -> Workload:
    """2D CPM, n x n lattice, Moore-8, periodic; one-pixel cells at distinct
    uniform random sites; target volume 100; J(cell,cell)=20,
    J(cell,medium)=10, lambda_V=50, no perimeter or Act term, T=20 (S=1)."""
    rng = np.random.default_rng(seed)
    lat = np.zeros((1, n, n), dtype=np.int32)
    sites = rng.choice(n * n, size=n_cells, replace=False)
    lat.reshape(-1)[sites] = np.arange(1, n_cells + 1, dtype=np.int32)
    J, lv, vt, lp, at, la, ma = _params()
    _sym(J, 1, 1, 20)
    _sym(J, 1, 0, 10)
    lv[1] = 50
    vt[1] = 100
    ct = np.ones(n_cells + 1, dtype=np.uint8)
    ct[0] = 0
    return Workload("cpm2d_%dx%d_moore8_%dcells" % (n, n, n_cells), 2, n, n, 1, J, lv, vt, lp,
                    at, la, ma, 20.0, 1, a, c, P, seed, 2, lat, ct, None, n_mcs)


def cube_cells_3d(seed: int = 1, n: int = 256, spacing: float = 10.0, a: int = 8, c: int = 2,
               P: int = 2, n_mcs: int = 1000) -> Workload:
    """3D CPM, n^3 lattice, 26-neighbourhood, periodic; 3^3 cubes at
    blue-noise centres (jittered grid, spacing 10, jitter 2: about 16,000
    cells at n=256); V_t=500, A_t=400; J(c,c)=20, J(c,m)=12, lambda_V=25,
    lambda_P=0.5, T=20, all scaled by S=2."""
    rng = np.random.default_rng(seed)
    lat = np.zeros((n, n, n), dtype=np.int32)
    ctr = jittered_centres((n, n, n), spacing, 2.0, rng)
    ctr = ctr[rng.permutation(len(ctr))]
    nc = place_cubes(lat, ctr, 3)
    S = 2
    J, lv, vt, lp, at, la, ma = _params()
    _sym(J, 1, 1, 20 * S)
    _sym(J, 1, 0, 12 * S)
    lv[1] = 25 * S
    vt[1] = 500
    lp[1] = 1            # 0.5 * S
    at[1] = 400
    ct = np.ones(nc + 1, dtype=np.uint8)
    ct[0] = 0
    return Workload("cpm3d_%d^3_moore26_%dcells" % (n, nc), 3, n, n, n, J, lv, vt, lp, at,
                    la, ma, 20.0 * S, S, a, c, P, seed, 2, lat, ct, None, n_mcs)


# Schedule of the 3D fibre tissue in the benchmark and its tests: areas of 16^3
# sites in a 2x2x2 checkerboard (blocks of 8^3), 64 colour cycles per MCS, 8
# rounds per colour visit.  Chosen by the statistical comparison with the
# serial chain at 128^3 (64 seeds, paired by seed): the paper's 4^3 areas
# raise the acceptance rate by 17% and the cell-volume variance by 40%, 8^3
# areas still raise the acceptance by about 1.3% and the variance or the MSD
# by 2-3% (about 1.6 concurrent attempts per 800-site cell per round), while
# 16^3 areas with 8 rounds per visit match every statistic within 1%.
TISSUE_SCHEDULE = {"a": 16, "c": 2, "P": 64}
# MCS of growth before the tissue is timed or compared: cells start as 3^3
# seeds and reach their target volume within about 20 MCS; the per-MCS cost
# settles by about 60.
TISSUE_BURN_IN = 60

# Target surface of the 3D fibre tissue.  The paper gives none for this workload; it is
# fixed at 1.2x the 26-neighbourhood interface count of a digital ball of about
# 800 voxels (radius 5.75: 799 voxels, 3,866 interfaces), i.e. 4,639.
TISSUE_A_TARGET = 4639


def fibre_mask(shape, rng, cell_spacing: float = 48.0, frac: float = 0.15,
               device: Optional[str] = None) -> np.ndarray:
    """Boolean mask of a Voronoi-edge 'fibre' network.

    Voronoi seeds sit on a jittered grid of the given spacing; a voxel lies on
    the network when its nearest and third-nearest seeds are almost equally
    far (it is close to a line where three Voronoi regions meet).  The
    closeness threshold is the ``frac`` quantile of that gap, so the mask
    freezes ``frac`` of the voxels.  Periodic.  Uses torch (on ``device`` if
    given) only to evaluate distances quickly."""
    import torch
    dev = torch.device(device or "cpu")
    shape = tuple(int(x) for x in shape)
    g = [max(4, int(round(n / cell_spacing))) for n in shape]
    step = [shape[d] / g[d] for d in range(3)]
    jit = rng.uniform(-0.4, 0.4, size=(g[0], g[1], g[2], 3))
    base = np.stack(np.meshgrid(*[np.arange(m) for m in g], indexing="ij"), axis=-1)
    seeds = (base + 0.5 + jit) * np.array(step)[None, None, None, :]
    seeds_t = torch.tensor(seeds, dtype=torch.float32, device=dev)
    nz, ny, nx = shape
    # candidate seeds: the 4x4x4 grid cells around each voxel's own cell
    offs = torch.tensor([(i, j, k) for i in range(-2, 2) for j in range(-2, 2) for k in range(-2, 2)],
                        device=dev)
    L = torch.tensor([nz, ny, nx], dtype=torch.float32, device=dev)
    gt = torch.tensor(g, device=dev)
    st = torch.tensor(step, dtype=torch.float32, device=dev)
    yy, xx = torch.meshgrid(torch.arange(ny, device=dev), torch.arange(nx, device=dev), indexing="ij")
    gap = torch.empty(shape, dtype=torch.float16, device=dev)
    zc = max(1, min(nz, (1 << 22) // (ny * nx)))
    for z0 in range(0, nz, zc):
        z1 = min(nz, z0 + zc)
        zz = torch.arange(z0, z1, device=dev)[:, None, None].expand(z1 - z0, ny, nx)
        p = torch.stack([zz, yy.expand_as(zz), xx.expand_as(zz)], dim=-1).float() + 0.5
        q = p / st
        cell = q.floor().long()
        shift = ((q - cell) >= 0.5).long()
        cand = cell[..., None, :] + offs + shift[..., None, :]
        ci = cand % gt
        sp = seeds_t[ci[..., 0], ci[..., 1], ci[..., 2]]
        d = sp - p[..., None, :]
        d = d - torch.round(d / L) * L
        dist = d.norm(dim=-1)
        top = torch.topk(dist, 3, dim=-1, largest=False).values
        gap[z0:z1] = (top[..., 2] - top[..., 0]).half()
    flat = gap.reshape(-1)
    gen = torch.Generator(device="cpu").manual_seed(int(rng.integers(1 << 31)))
    idx = torch.randint(0, flat.numel(), (min(flat.numel(), 1 << 22),), generator=gen).to(dev)
    thr = torch.quantile(flat[idx].float(), frac)
    return (gap < thr.half()).cpu().numpy()


def fibre_tissue_3d(seed: int = 1, n: int = 1024, a: int = 8, c: int = 2, P: int = 2,
               n_mcs: int = 200, device: Optional[str] = None,
               fibre_spacing: float = 48.0) -> Workload:
    """3D tissue-scale CPM with a frozen Voronoi-edge fibre network (about 15%
    of voxels) and motile cells (Act model on).  Cells start as 3^3 cubes at
    blue-noise centres (spacing 10) outside the fibres; V_t=800; Act:
    lambda_act=200, Max_act=30; J(c,c)=20, J(c,medium)=10, J(c,fibre)=40,
    lambda_V=25, lambda_P=0.2, T=20, all scaled by S=5."""
    rng = np.random.default_rng(seed)
    shape = (n, n, n)
    # at least 4 Voronoi seeds per axis, so the 4x4x4 candidate window never wraps onto itself
    fib = fibre_mask(shape, rng, cell_spacing=min(fibre_spacing, n / 4), device=device)
    lat = np.zeros(shape, dtype=np.int32)
    lat[fib] = -1
    ctr = jittered_centres(shape, 10.0, 2.0, rng)
    ok = ~fib[ctr[:, 0], ctr[:, 1], ctr[:, 2]]
    ctr = ctr[ok]
    ctr = ctr[rng.permutation(len(ctr))]
    nc = place_cubes(lat, ctr, 3)
    S = 5
    J, lv, vt, lp, at, la, ma = _params()
    _sym(J, 1, 1, 20 * S)
    _sym(J, 1, 0, 10 * S)
    _sym(J, 1, 2, 40 * S)
    lv[1] = 25 * S
    vt[1] = 800
    lp[1] = 1            # 0.2 * S
    at[1] = TISSUE_A_TARGET
    la[1] = 200 * S
    ma[1] = 30
    ct = np.ones(nc + 1, dtype=np.uint8)
    ct[0] = 0
    return Workload("cpm3d_tissue_%d^3_act_fibre_%dcells" % (n, nc), 3, n, n, n, J, lv, vt,
                    lp, at, la, ma, 20.0 * S, S, a, c, P, seed, 2, lat, ct, None, n_mcs)


def random_small(seed: int, dim: int = 2, n: int = 16, n_cells: int = 6, edge: int = 3,
                 perimeter: bool = True, act: bool = False, obstacles: float = 0.0,
                 a: Optional[int] = None, c: int = 2, P: int = 1, T: float = 20.0,
                 n_types: int = 2) -> Workload:
    """Small randomised lattices for unit tests: cubes (squares) of random
    types at random centres, optional obstacle sites and Act values, and
    random integer parameters of the magnitudes the paper's tables use."""
    rng = np.random.default_rng(seed)
    shape = (n,) * dim
    lat = np.zeros(shape, dtype=np.int32)
    if obstacles > 0:
        lat[rng.random(shape) < obstacles] = -1
    ctr = rng.integers(0, n, size=(n_cells, dim))
    nc = place_cubes(lat, ctr, edge)
    J, lv, vt, lp, at, la, ma = _params()
    obstacle_type = n_types + 1
    for t1 in range(0, obstacle_type + 1):
        for t2 in range(t1, obstacle_type + 1):
            if t1 == 0 and t2 == 0:
                continue
            _sym(J, t1, t2, int(rng.integers(0, 40)))
    for t in range(1, n_types + 1):
        lv[t] = int(rng.integers(1, 60))
        vt[t] = int(rng.integers(4, max(5, 4 * edge ** dim)))
        if perimeter:
            lp[t] = int(rng.integers(1, 4))
            at[t] = int(rng.integers(4, 8 * edge ** (dim - 1) * (3 if dim == 3 else 2)))
        if act:
            la[t] = int(rng.integers(50, 800))
            ma[t] = int(rng.integers(5, 60))
    ct = np.zeros(nc + 1, dtype=np.uint8)
    ct[1:] = rng.integers(1, n_types + 1, size=nc)
    actv = None
    if act:
        actv = np.zeros(shape, dtype=np.uint8)
        cells = lat > 0
        mx = ma[ct[np.maximum(lat, 0)]]
        draw = rng.integers(0, 61, size=shape)
        actv[cells] = np.minimum(draw[cells], mx[cells]).astype(np.uint8)
    if a is None:
        a = 4
    if dim == 2:
        lat = lat[None]
        if actv is not None:
            actv = actv[None]
    nz = 1 if dim == 2 else n
    return Workload("random_small_%dd_%d" % (dim, seed), dim, n, n, nz, J, lv, vt, lp, at, la,
                    ma, float(T), 1, a, c, P, seed, obstacle_type, lat, ct, actv, 1)


# --------------------------------------------------------------------------
# an ensemble for parameter sweeps
# --------------------------------------------------------------------------

SWEEP_RANGES = {            # the seven swept parameters, in model units
    "J_cc": (5.0, 40.0),
    "J_cm": (2.0, 25.0),
    "lambda_V": (5.0, 100.0),
    "lambda_P": (0.0, 2.0),
    "lambda_act": (0.0, 400.0),
    "max_act": (10.0, 60.0),
    "T": (5.0, 40.0),
}
SWEEP_SCALE = 10            # integer energy scale S for the swept parameters


def latin_hypercube(n: int, rng) -> dict:
    """n points of a Latin hypercube over SWEEP_RANGES: every parameter's
    range is cut into n strata, each used once, in an independent random
    order, with a uniform position inside the stratum."""
    out = {}
    for k, (lo, hi) in SWEEP_RANGES.items():
        u = (rng.permutation(n) + rng.random(n)) / n
        out[k] = lo + (hi - lo) * u
    return out


def ensemble(n: int = 512, seed: int = 1, dim: Optional[int] = None, side2=(64, 512), side3=(64, 128),
             cells=(10, 2000), a: int = 4, c: int = 2) -> list:
    """Parameter-sweep ensemble: n lattices of uneven sizes (log-uniform edge, 2D or 3D),
    10..2000 cells each, parameters from a Latin hypercube (SWEEP_RANGES,
    scaled by SWEEP_SCALE).  Targets: V_t = half the lattice per cell (at
    least 10 sites); A_t = 1.2x an estimate of a compact cell's interface
    count (12.5 sqrt(V) in 2D with 8 neighbours, 45 V^(2/3) in 3D with 26).
    Cells start as squares / cubes of edge 3 at jittered-grid centres."""
    rng = np.random.default_rng(seed)
    hc = latin_hypercube(n, rng)
    S = SWEEP_SCALE
    out = []
    for k in range(n):
        d = dim if dim is not None else int(rng.integers(2, 4))
        lo, hi = side2 if d == 2 else side3
        side = int(np.exp(rng.uniform(np.log(lo), np.log(hi))))
        side = max(8 * a, (side // (2 * a)) * (2 * a))
        shape = (side,) * d
        n_sites = side ** d
        nc = int(np.exp(rng.uniform(np.log(cells[0]), np.log(cells[1]))))
        nc = max(1, min(nc, n_sites // 64))
        spacing = (n_sites / nc) ** (1.0 / d)
        lat = np.zeros(shape, dtype=np.int32)
        ctr = jittered_centres(shape, spacing, max(0.0, spacing / 2 - 2), rng)
        ctr = ctr[rng.permutation(len(ctr))][:nc]
        ncell = place_cubes(lat, ctr, 3)
        J, lv, vt, lp, at, la, ma = _params()
        _sym(J, 1, 1, int(round(hc["J_cc"][k] * S)))
        _sym(J, 1, 0, int(round(hc["J_cm"][k] * S)))
        lv[1] = int(round(hc["lambda_V"][k] * S))
        v_t = max(10, int(0.5 * n_sites / max(ncell, 1)))
        vt[1] = v_t
        lp[1] = int(round(hc["lambda_P"][k] * S))
        at[1] = int(round(1.2 * (12.5 * v_t ** 0.5 if d == 2 else 45.0 * v_t ** (2.0 / 3.0))))
        la[1] = int(round(hc["lambda_act"][k] * S))
        ma[1] = int(round(hc["max_act"][k]))
        ct = np.ones(ncell + 1, dtype=np.uint8)
        ct[0] = 0
        if d == 2:
            lat = lat[None]
        P = (a // c) ** d  # one round per colour visit
        out.append(Workload("ensemble_%d_%dd_%d" % (k, d, side), d, side, side, 1 if d == 2 else side, J, lv, vt,
                            lp, at, la, ma, float(hc["T"][k] * S), S, a, c, P, seed * 100003 + k, 2, lat, ct,
                            None, 1000))
    return out


# --------------------------------------------------------------------------
# inputs of the emulator (swept parameters, network initialisation)
# --------------------------------------------------------------------------

EMULATOR_PARAMS = list(SWEEP_RANGES)      # input order of the emulator
EMULATOR_SIDE = 64                         # 2D lattice edge of every emulator run
EMULATOR_CELLS = 16                        # cells per run (V_t = half the lattice per cell = 128)


def sweep_points(n: int, seed: int) -> np.ndarray:
    """n parameter points [n, 7] (model units, EMULATOR_PARAMS order) from a
    seeded Latin hypercube over SWEEP_RANGES, rounded to the integer grid
    the CPM simulates (energies x SWEEP_SCALE, Max_Act to whole MCS)."""
    hc = latin_hypercube(n, np.random.default_rng(seed))
    X = np.stack([hc[k] for k in EMULATOR_PARAMS], axis=1)
    S = SWEEP_SCALE
    X = np.round(X * S) / S
    X[:, EMULATOR_PARAMS.index("max_act")] = np.round(X[:, EMULATOR_PARAMS.index("max_act")])
    return X


def scale_inputs(X) -> np.ndarray:
    """Min-max scaling of parameter points to [0, 1] over SWEEP_RANGES."""
    lo = np.array([SWEEP_RANGES[k][0] for k in EMULATOR_PARAMS])
    hi = np.array([SWEEP_RANGES[k][1] for k in EMULATOR_PARAMS])
    return ((np.asarray(X, dtype=np.float64) - lo) / (hi - lo)).astype(np.float32)


def emulator_run(theta, seed: int, side: int = EMULATOR_SIDE, n_cells: int = EMULATOR_CELLS, a: int = 4,
                 c: int = 2) -> Workload:
    """One run of the emulator's training set: a 2D side x side periodic
    lattice, Moore neighbourhood, n_cells cells started as 3 x 3 squares at
    jittered-grid centres (the ensemble recipe at fixed size and cell count),
    parameters theta (model units, EMULATOR_PARAMS order), S = SWEEP_SCALE,
    the ensemble's checkerboard (a x a areas, c x c colours, one round per
    colour visit).  The seed fixes the start and the Philox key."""
    rng = np.random.default_rng(seed)
    th = dict(zip(EMULATOR_PARAMS, np.asarray(theta, dtype=np.float64)))
    shape = (side, side)
    spacing = (side * side / n_cells) ** 0.5
    lat = np.zeros(shape, dtype=np.int32)
    ctr = jittered_centres(shape, spacing, max(0.0, spacing / 2 - 2), rng)
    ctr = ctr[rng.permutation(len(ctr))][:n_cells]
    ncell = place_cubes(lat, ctr, 3)
    S = SWEEP_SCALE
    J, lv, vt, lp, at, la, ma = _params()
    _sym(J, 1, 1, int(round(th["J_cc"] * S)))
    _sym(J, 1, 0, int(round(th["J_cm"] * S)))
    lv[1] = int(round(th["lambda_V"] * S))
    v_t = max(10, int(0.5 * side * side / max(ncell, 1)))
    vt[1] = v_t
    lp[1] = int(round(th["lambda_P"] * S))
    at[1] = int(round(1.2 * 12.5 * v_t ** 0.5))
    la[1] = int(round(th["lambda_act"] * S))
    ma[1] = int(round(th["max_act"]))
    ct = np.ones(ncell + 1, dtype=np.uint8)
    ct[0] = 0
    return Workload("emulator_%d" % seed, 2, side, side, 1, J, lv, vt, lp, at, la, ma, float(th["T"] * S), S, a, c,
                    (a // c) ** 2, seed, 2, lat[None], ct, None, 1)


def mlp_init(seed: int, n_members: int, sizes) -> np.ndarray:
    """Initial parameters of an MLP ensemble, flat float32 [n_members, P] in
    the layout W_1 [out][in], b_1, W_2, b_2, ...: weights N(0, 2/fan_in)
    (He et al. 2015), biases zero; each member from its own stream."""
    out = []
    for e in range(n_members):
        rng = np.random.default_rng([seed, e])
        parts = []
        for i, o in zip(sizes[:-1], sizes[1:]):
            parts.append(rng.normal(0.0, (2.0 / i) ** 0.5, (o, i)).ravel())
            parts.append(np.zeros(o))
        out.append(np.concatenate(parts))
    return np.asarray(out, dtype=np.float32)


# --------------------------------------------------------------------------
# cell sorting (two cell types with differential adhesion)
# --------------------------------------------------------------------------

def sorting_2d(seed: int = 1, n: int = 128, edge: int = 8, a: int = 4, c: int = 2, P: int = 1) -> Workload:
    """Cell sorting by differential adhesion (Results, Fig. 4, after Graner &
    Glazier): a confluent 2D n x n periodic tissue, Moore-8, tiled by
    edge x edge square cells (no medium), each cell type 1 ("dark") or 2
    ("light") at random in equal numbers; J(d,d) = 2, J(l,l) = 14,
    J(l,d) = 11, J with the medium 16, V_t = edge^2, lambda_V = 1, T = 10."""
    rng = np.random.default_rng(seed)
    k = n // edge
    n_cells = k * k
    ids = np.arange(1, n_cells + 1, dtype=np.int32).reshape(k, k)
    lat = np.repeat(np.repeat(ids, edge, axis=0), edge, axis=1)[None]
    types = np.array([1] * (n_cells // 2) + [2] * (n_cells - n_cells // 2), dtype=np.uint8)
    rng.shuffle(types)
    ct = np.concatenate([[0], types]).astype(np.uint8)
    J, lv, vt, lp, at, la, ma = _params()
    _sym(J, 1, 1, 2)
    _sym(J, 2, 2, 14)
    _sym(J, 1, 2, 11)
    _sym(J, 0, 1, 16)
    _sym(J, 0, 2, 16)
    for t in (1, 2):
        lv[t] = 1
        vt[t] = edge * edge
    return Workload("sorting_%d" % seed, 2, n, n, 1, J, lv, vt, lp, at, la, ma, 10.0, 1, a, c, P, seed, 3, lat, ct,
                    None, 1)


# --------------------------------------------------------------------------
# motility fields and settings (Eq. 4 to Eq. 7)
# --------------------------------------------------------------------------

def circular_field(nx: int, ny: int, nz: int = 1, dim: int = 2) -> np.ndarray:
    """The paper's 2D chemotaxis field (Table 1, Fig. 6A): unit vectors at
    90 degrees to the radial vector from the lattice centre (a circular
    flow), in Q14 int16 components; the same in every z plane for 3D (z
    component 0); the centre site gets (0, 0)."""
    y, x = np.mgrid[0:ny, 0:nx].astype(np.float64)
    rx, ry = x - (nx - 1) / 2.0, y - (ny - 1) / 2.0
    r = np.hypot(rx, ry)
    with np.errstate(invalid="ignore", divide="ignore"):
        vx = np.where(r > 0, -ry / r, 0.0)
        vy = np.where(r > 0, rx / r, 0.0)
    f = np.zeros((nz, ny, nx, dim), dtype=np.int16)
    f[..., 0] = np.round(vx * 16384).astype(np.int16)[None]
    f[..., 1] = np.round(vy * 16384).astype(np.int16)[None]
    return f


def uniform_field(shape, dim: int, direction) -> np.ndarray:
    """A constant field of unit vectors along ``direction`` (Q14 int16)."""
    d = np.asarray(direction, dtype=np.float64)
    d = d / np.linalg.norm(d)
    f = np.zeros(tuple(shape) + (dim,), dtype=np.int16)
    for k in range(dim):
        f[..., k] = int(round(d[k] * 16384))
    return f


def with_motility(w: Workload, chem=None, lambda_chem=0, lambda_pers=0, mu=0.0, dt=1, types=None) -> Workload:
    """w with the chemotaxis field ``chem`` (or None) and the same
    lambda_chem, lambda_pers, mu and dt for every cell type in ``types``
    (all cell types by default)."""
    types = range(1, MAX_TYPES) if types is None else types
    lc = np.zeros(MAX_TYPES, dtype=np.int32)
    lp = np.zeros(MAX_TYPES, dtype=np.int32)
    mu_ = np.zeros(MAX_TYPES, dtype=np.float64)
    dt_ = np.zeros(MAX_TYPES, dtype=np.int32)
    for t in types:
        lc[t], lp[t], mu_[t], dt_[t] = lambda_chem, lambda_pers, mu, dt
    return w.replace(chem_field=chem, lambda_chem=lc if chem is not None else None,
                     lambda_pers=lp if lambda_pers else None, mu_pers=mu_ if lambda_pers else None,
                     dt_pers=dt_ if lambda_pers else None)
