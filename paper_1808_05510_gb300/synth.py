"""Seeded synthetic problem generators for the smoothed connectome regression.

This module produces the *inputs* of the greedy solver (Algorithm 1's input
line): the voxel masks, the graph Laplacians ``L_x``/``L_y`` of the voxel
face-adjacency graphs (Sec. 1.1: unit weights, free boundary at the mask edge),
the injection matrix ``X``, the projection matrix ``Y``, the observation mask
``Omega`` and ``lambda``.  It contains none of the solver's arithmetic, so the
oracle and the CUDA path can both consume it without sharing method code.

The recipes stand in for the Allen top-view / flatmap data and the paper's toy
brain (Sec. 3.1), which are not available: every workload is synthetic, with
the shapes, injection statistics and mask structure of the paper's problems.

* Injection ``alpha``: centre drawn uniformly among mask voxels, Gaussian blob
  ``X_k,alpha = A exp(-|p_k - c|^2 / (2 sigma^2))`` (distances in voxels),
  truncated to zero beyond ``3 sigma`` (so ``X`` is sparse).
* ``Omega_i,alpha = 1{X_i,alpha <= 0.4}`` -- unobserved on the injection site
  (Sec. 4 data description uses the 0.4 threshold; 1 = observed).
* ``W_true(p_i, p_k) = exp(-|p_i - p_k|^2/0.4^2)
  + 0.9 exp(-(|p_k - a|^2 + |p_i - b|^2)/0.2^2)``, ``a = 0.8*1``,
  ``b = 0.1*1`` in coordinates normalised to ``[0,1]^d``: the d-dimensional
  restatement of the toy kernel, Eq. (W_true_toy), read with the first
  argument the target and the second the source.
* ``Y = (W_true X + eps) o Omega`` with ``eps ~ N(0, (0.01 max|W_true X o Omega|)^2)``.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional, Tuple

import numpy as np


@dataclasses.dataclass
class Grid:
    """A voxel region: a boolean mask inside a box, active voxels numbered in
    C (row-major) order of the box."""

    mask: np.ndarray  # bool, box shape (d0, d1[, d2])

    @property
    def n(self) -> int:
        return int(self.mask.sum())

    def coords(self) -> np.ndarray:
        """(n, d) integer voxel coordinates of the active voxels."""
        return np.argwhere(self.mask)

    def unit_coords(self) -> np.ndarray:
        """(n, d) coordinates normalised per axis to [0, 1]."""
        c = self.coords().astype(np.float64)
        dims = np.array(self.mask.shape, dtype=np.float64)
        return c / np.maximum(dims - 1.0, 1.0)


@dataclasses.dataclass
class CSR:
    """Square sparse matrix in CSR form with int32 indices and float64 values."""

    n: int
    rowptr: np.ndarray  # int32 (n+1)
    col: np.ndarray  # int32 (nnz)
    val: np.ndarray  # float64 (nnz)

    def to_dense(self) -> np.ndarray:
        A = np.zeros((self.n, self.n))
        for i in range(self.n):
            for p in range(self.rowptr[i], self.rowptr[i + 1]):
                A[i, self.col[p]] += self.val[p]
        return A


@dataclasses.dataclass
class Problem:
    """Inputs of Algorithm 1 (all float64 unless stated)."""

    name: str
    grid_x: Grid
    grid_y: Grid
    Lx: CSR
    Ly: CSR
    X: np.ndarray  # (nx, m) column-major semantics, stored as a numpy array
    Y: np.ndarray  # (ny, m)
    Omega: np.ndarray  # (ny, m) uint8, 1 = observed
    lam: float
    r_max: int
    W_true: Optional[np.ndarray] = None  # dense only for tiny problems

    @property
    def nx(self) -> int:
        return self.X.shape[0]

    @property
    def ny(self) -> int:
        return self.Y.shape[0]

    @property
    def m(self) -> int:
        return self.X.shape[1]


# ----------------------------------------------------------------------------
# Laplacian of the face-adjacency graph (problem data, Sec. 1.1)
# ----------------------------------------------------------------------------

def grid_laplacian(grid: Grid) -> CSR:
    """Graph Laplacian ``Deg - Adj`` of the face-adjacency graph of the active
    voxels, unit edge weights, free (Neumann) at the mask boundary; columns of
    each row sorted ascending (the diagonal included)."""
    mask = grid.mask
    shape = mask.shape
    index = -np.ones(shape, dtype=np.int64)
    coords = np.argwhere(mask)
    n = coords.shape[0]
    index[tuple(coords.T)] = np.arange(n)
    nbrs = []
    for ax in range(mask.ndim):
        for step in (-1, 1):
            c = coords.copy()
            c[:, ax] += step
            ok = (c[:, ax] >= 0) & (c[:, ax] < shape[ax])
            j = -np.ones(n, dtype=np.int64)
            j[ok] = index[tuple(c[ok].T)]
            nbrs.append(j)
    nbrs = np.stack(nbrs, axis=1)  # (n, 2d)
    deg = (nbrs >= 0).sum(axis=1)
    # each row: the diagonal (i, deg_i) and (i, j, -1) for every face neighbour j,
    # columns ascending.  Indices follow the row-major voxel order, so the face
    # neighbours of i sort as -axis0 < ... < -axis_last < i < +axis_last < ... < +axis0.
    d = mask.ndim
    order = [2 * ax for ax in range(d)] + [-1] + [2 * ax + 1 for ax in reversed(range(d))]
    ent = np.stack([np.arange(n) if k < 0 else nbrs[:, k] for k in order], axis=1)
    keep = ent >= 0
    cols = ent[keep]
    rows = np.broadcast_to(np.arange(n)[:, None], ent.shape)[keep]
    vals = np.where(cols == rows, deg[rows].astype(np.float64), -1.0)
    rowptr = np.concatenate([[0], np.cumsum(keep.sum(axis=1))]).astype(np.int32)
    return CSR(n, rowptr, np.asarray(cols, dtype=np.int32), np.asarray(vals, dtype=np.float64))


# ----------------------------------------------------------------------------
# Masks
# ----------------------------------------------------------------------------

def _largest_component(mask: np.ndarray) -> np.ndarray:
    from scipy import ndimage

    lab, k = ndimage.label(mask)  # default structure = face connectivity
    if k == 0:
        return mask
    sizes = np.bincount(lab.ravel())
    sizes[0] = 0
    return lab == int(np.argmax(sizes))


def blob_mask(shape, target: int, rng: np.random.Generator, smooth: float = 4.0) -> np.ndarray:
    """Smoothed Gaussian random field thresholded for about ``target`` voxels,
    then restricted to its largest face-connected component."""
    from scipy import ndimage

    field = ndimage.gaussian_filter(rng.standard_normal(shape), smooth, mode="constant")
    lo, hi = 0.0, 1.0
    mask = None
    for _ in range(40):  # bisection on the quantile so the component has ~target voxels
        q = 0.5 * (lo + hi)
        thr = np.quantile(field, 1.0 - q)
        mask = _largest_component(field > thr)
        cnt = int(mask.sum())
        if abs(cnt - target) <= max(1, target // 200):
            break
        if cnt < target:
            lo = q
        else:
            hi = q
    return mask


def shell_mask(shape, target: int) -> np.ndarray:
    """Ellipsoidal shell: outer semi-axes 0.46*dims, thickness bisected so the
    shell holds about ``target`` voxels (largest face-connected component)."""
    dims = np.array(shape, dtype=np.float64)
    ctr = (dims - 1.0) / 2.0
    ax = 0.46 * dims
    g = np.stack(np.meshgrid(*[np.arange(s) for s in shape], indexing="ij"), axis=-1).astype(np.float64)
    rho_out = np.sqrt((((g - ctr) / ax) ** 2).sum(-1))
    lo, hi = 0.0, 1.0
    mask = None
    for _ in range(60):
        t = 0.5 * (lo + hi)  # fractional thickness
        mask = _largest_component((rho_out <= 1.0) & (rho_out >= 1.0 - t))
        cnt = int(mask.sum())
        if abs(cnt - target) <= max(1, target // 200):
            break
        if cnt < target:
            lo = t
        else:
            hi = t
    return mask


# ----------------------------------------------------------------------------
# Injections, W_true, Y
# ----------------------------------------------------------------------------

def gaussian_injections(grid: Grid, m: int, rng: np.random.Generator, sigma_lo: float, sigma_hi: float,
                        amp_lo: float, amp_hi: float) -> np.ndarray:
    """Dense (n, m) X of truncated Gaussian blobs centred on random mask voxels."""
    c = grid.coords().astype(np.float64)
    n = c.shape[0]
    X = np.zeros((n, m))
    for a in range(m):
        ctr = c[rng.integers(n)]
        sig = rng.uniform(sigma_lo, sigma_hi) if sigma_hi > sigma_lo else sigma_lo
        amp = rng.uniform(amp_lo, amp_hi) if amp_hi > amp_lo else amp_lo
        d2 = ((c - ctr) ** 2).sum(1)
        col = amp * np.exp(-d2 / (2.0 * sig * sig))
        col[d2 > (3.0 * sig) ** 2] = 0.0
        X[:, a] = col
    return X


def w_true_block(py: np.ndarray, px: np.ndarray, sparse_cut: float = 0.0) -> np.ndarray:
    """W_true(p_i, p_k) for target points ``py`` (rows) and source points ``px``."""
    d = py.shape[1]
    a = 0.8 * np.ones(d)
    b = 0.1 * np.ones(d)
    d2 = (py * py).sum(1)[:, None] + (px * px).sum(1)[None, :] - 2.0 * (py @ px.T)
    np.maximum(d2, 0.0, out=d2)
    w = np.exp(-d2 / 0.16)
    w += 0.9 * np.exp(-(((px - a) ** 2).sum(-1)[None, :] + ((py - b) ** 2).sum(-1)[:, None]) / 0.04)
    if sparse_cut > 0.0:
        w[w < sparse_cut] = 0.0
    return w


def make_Y(grid_y: Grid, grid_x: Grid, X: np.ndarray, Omega: np.ndarray, rng: np.random.Generator,
           noise_rel: float, sparse_cut: float = 0.0, chunk: int = 4096) -> np.ndarray:
    """Y = (W_true X + eps) o Omega, W_true applied tile-wise over the support of X."""
    py = grid_y.unit_coords()
    px = grid_x.unit_coords()
    supp = np.flatnonzero(np.any(X != 0.0, axis=1))
    Xs = X[supp]
    pxs = px[supp]
    WX = np.zeros((py.shape[0], X.shape[1]))
    for s in range(0, py.shape[0], chunk):
        WX[s:s + chunk] = w_true_block(py[s:s + chunk], pxs, sparse_cut) @ Xs
    scale = noise_rel * np.max(np.abs(WX * Omega))
    eps = rng.standard_normal(WX.shape) * scale
    return (WX + eps) * Omega


def _finish(name, grid_x, grid_y, X, rng, lam, r_max, noise_rel=0.01, sparse_cut=0.0, omega_from_x=True,
            keep_w_true=False):
    if omega_from_x:
        # Same grid for source and target (nx = ny): the injection site is unobserved.
        Omega = (X <= 0.4).astype(np.uint8)
    else:
        Omega = np.ones((grid_y.n, X.shape[1]), dtype=np.uint8)
    Y = make_Y(grid_y, grid_x, X, Omega, rng, noise_rel, sparse_cut)
    W_true = None
    if keep_w_true:
        W_true = w_true_block(grid_y.unit_coords(), grid_x.unit_coords(), sparse_cut)
    return Problem(name, grid_x, grid_y, grid_laplacian(grid_x), grid_laplacian(grid_y), X, Y, Omega,
                   float(lam), int(r_max), W_true)


# ----------------------------------------------------------------------------
# Workloads
# ----------------------------------------------------------------------------

def toy2d(seed: int = 1809, side: int = 20, m: int = 5, lam: float = 100.0, r_max: int = 20) -> Problem:
    """Toy plain-FP64 workload: 20x20 grid, 5-point Laplacian, 5 blobs (sigma 2 voxels)."""
    rng = np.random.default_rng(seed)
    g = Grid(np.ones((side, side), dtype=bool))
    X = gaussian_injections(g, m, rng, 2.0, 2.0, 1.0, 1.0)
    return _finish(f"toy2d-{side}x{side}-m{m}", g, g, X, rng, lam, r_max, keep_w_true=True)


def visual_cortex(seed: int = 1810, box: int = 40, n_target: int = 7500, m: int = 28, lam: float = 1e2,
                  r_max: int = 100) -> Problem:
    """Visual-cortex-shaped workload: ~7,500 voxels of a smooth random blob in a 40^3 box,
    7-point Laplacian, 28 blobs (sigma 2 voxels)."""
    rng = np.random.default_rng(seed)
    g = Grid(blob_mask((box, box, box), n_target, rng))
    X = gaussian_injections(g, m, rng, 2.0, 2.0, 1.0, 1.0)
    return _finish(f"visual-{g.n}vox-m{m}-lam{lam:g}", g, g, X, rng, lam, r_max)


def whole_cortex(seed: int = 1811, shape=(96, 64, 80), n_target: int = 45000, m: int = 126, lam: float = 1e3,
                 r_max: int = 500) -> Problem:
    """Whole-cortex-shaped workload: ellipsoidal shell of ~45,000 voxels in a 96x64x80 box,
    126 blobs (sigma 2..5 voxels, amplitude 0.2..1), W_true cut below 1e-3."""
    rng = np.random.default_rng(seed)
    g = Grid(shell_mask(shape, n_target))
    X = gaussian_injections(g, m, rng, 2.0, 5.0, 0.2, 1.0)
    return _finish(f"cortex-{g.n}vox-m{m}", g, g, X, rng, lam, r_max, sparse_cut=1e-3)


def stress_shell(seed: int = 1816, side: int = 256, n_target: int = 4_000_000, m: int = 8,
                 lam: float = 1e3) -> Problem:
    """Roofline stress shape: an ellipsoidal shell of ~4M voxels in a 256^3 box
    (outer semi-axes 0.46 side, thickness from the shell volume
    V (1 - (1 - t)^3) = n_target), 7-point Laplacian, m Gaussian injections,
    Omega = 1{X <= 0.4}, Y random on Omega (only the sub-solves run on it)."""
    rng = np.random.default_rng(seed)
    a = 0.46 * side
    vol = 4.0 / 3.0 * math.pi * a ** 3
    t = 1.0 - (1.0 - min(0.999, n_target / vol)) ** (1.0 / 3.0)
    c = (side - 1) / 2.0
    z, y, x = np.ogrid[:side, :side, :side]
    rho2 = ((z - c) / a) ** 2 + ((y - c) / a) ** 2 + ((x - c) / a) ** 2
    mask = (rho2 <= 1.0) & (rho2 >= (1.0 - t) ** 2)
    g = Grid(mask)
    X = gaussian_injections(g, m, rng, 2.0, 3.0, 1.0, 1.0)
    Omega = (X <= 0.4).astype(np.uint8)
    Y = rng.standard_normal((g.n, m)) * Omega
    L = grid_laplacian(g)
    return Problem(f"stress-shell-{g.n}vox-m{m}", g, g, L, L, X, Y, Omega, float(lam), 2)


def sweep_cortex(seed: int = 1814, box: int = 40, n_target: int = 15000, m: int = 126, lam: float = 1e2,
                 r_max: int = 200) -> Problem:
    """Data set of the lambda x fold sweep: the visual-cortex recipe on ~15,000
    voxels of a 40^3 box with 126 injections (each sweep member fits a subset)."""
    rng = np.random.default_rng(seed)
    g = Grid(blob_mask((box, box, box), n_target, rng))
    X = gaussian_injections(g, m, rng, 2.0, 2.0, 1.0, 1.0)
    return _finish(f"sweep-{g.n}vox-m{m}", g, g, X, rng, lam, r_max)


def fold_partition(m: int, k: int = 5, lo: int = 20, hi: int = 30, seed: int = 1815) -> List[np.ndarray]:
    """Seeded partition of the injections 0..m-1 into k folds whose sizes lie in
    [lo, hi] (uneven: the sizes are drawn, not equal)."""
    if not (k * lo <= m <= k * hi):
        raise ValueError("no partition with these fold sizes")
    rng = np.random.default_rng(seed)
    sizes = np.full(k, lo)
    for _ in range(m - k * lo):
        room = np.flatnonzero(sizes < hi)
        sizes[rng.choice(room)] += 1
    perm = rng.permutation(m)
    cuts = np.concatenate([[0], np.cumsum(sizes)])
    return [np.sort(perm[cuts[f]:cuts[f + 1]]) for f in range(k)]


def lambda_grid(count: int = 16, lo: float = 1e0, hi: float = 1e6) -> np.ndarray:
    """Log-spaced lambda values of the sweep."""
    return np.logspace(np.log10(lo), np.log10(hi), count)


def sweep_members(m: int, lams, folds) -> List[Tuple[float, np.ndarray, np.ndarray]]:
    """(lambda, fit columns, held-out columns) for every lambda x fold pair."""
    out = []
    for lam in lams:
        for test in folds:
            fit = np.setdiff1d(np.arange(m), test)
            out.append((float(lam), fit, np.asarray(test)))
    return out


def member_problem(p: Problem, lam: float, fit) -> Problem:
    """The sub-problem a sweep member solves: the fit columns of X, Y, Omega with its lambda."""
    fit = np.asarray(fit)
    return dataclasses.replace(p, name=f"{p.name}-lam{lam:g}-fit{len(fit)}", X=p.X[:, fit], Y=p.Y[:, fit],
                               Omega=p.Omega[:, fit], lam=float(lam))


def rect2d(seed: int = 1812, shape_y=(9, 7), shape_x=(6, 8), m: int = 4, lam: float = 3.0, r_max: int = 12,
           sigma: float = 1.2) -> Problem:
    """Tiny problem with different source and target grids (ny != nx) and a general
    random Omega, used to catch transposed operands."""
    rng = np.random.default_rng(seed)
    gy = Grid(np.ones(shape_y, dtype=bool))
    gx = Grid(np.ones(shape_x, dtype=bool))
    X = gaussian_injections(gx, m, rng, sigma, sigma, 0.5, 1.0)
    Omega = (rng.random((gy.n, m)) > 0.25).astype(np.uint8)
    Y = make_Y(gy, gx, X, Omega, rng, 0.01)
    return Problem(f"rect-{gy.n}x{gx.n}-m{m}", gx, gy, grid_laplacian(gx), grid_laplacian(gy), X, Y, Omega,
                   float(lam), int(r_max), w_true_block(gy.unit_coords(), gx.unit_coords()))


def masked3d(seed: int = 1813, box: int = 12, n_target: int = 700, m: int = 6, lam: float = 50.0,
             r_max: int = 30) -> Problem:
    """Small 3-D blob-mask problem (7-point Laplacian, irregular degrees) for parity tests."""
    rng = np.random.default_rng(seed)
    g = Grid(blob_mask((box, box, box), n_target, rng, smooth=2.0))
    X = gaussian_injections(g, m, rng, 1.5, 1.5, 1.0, 1.0)
    return _finish(f"masked3d-{g.n}vox-m{m}", g, g, X, rng, lam, r_max)


def box3d(seed: int = 1817, side: int = 50, m: int = 2, lam: float = 50.0, r_max: int = 4) -> Problem:
    """Full side^3 box (every voxel active, 7-point Laplacian) with m blobs (sigma 2 voxels):
    a large single-cluster case (125,000 rows at side 50)."""
    rng = np.random.default_rng(seed)
    g = Grid(np.ones((side, side, side), dtype=bool))
    X = gaussian_injections(g, m, rng, 2.0, 2.0, 1.0, 1.0)
    return _finish(f"box{side}-m{m}", g, g, X, rng, lam, r_max)


def paper_toy(seed: int = 1808, n: int = 200, m: int = 5, lam: float = 100.0, noise: float = 0.1,
              quadrature: bool = False) -> Problem:
    """The paper's 1-D toy brain (Sec. 3.1): n-point chain on [0, 1], m box injections of
    width 0.12 + 0.1*U(0,1), X = 1 inside the box, Omega = 1 - X, Gaussian noise of
    standard deviation ``noise``.  ``quadrature`` multiplies W_true X by 1/n."""
    rng = np.random.default_rng(seed)
    g = Grid(np.ones((n,), dtype=bool))
    x = g.unit_coords()[:, 0]
    X = np.zeros((n, m))
    for a in range(m):
        width = 0.12 + 0.1 * rng.random()
        c = rng.uniform(width / 2, 1.0 - width / 2)
        X[:, a] = (np.abs(x - c) <= width / 2).astype(np.float64)
    Omega = (1.0 - X).astype(np.uint8)
    W = w_true_block(g.unit_coords(), g.unit_coords())
    WX = W @ X * ((1.0 / n) if quadrature else 1.0)
    Y = (WX + noise * rng.standard_normal(WX.shape)) * Omega
    return Problem(f"paper-toy-n{n}", g, g, grid_laplacian(g), grid_laplacian(g), X, Y, Omega, float(lam), 140, W)


WORKLOADS = {
    "toy2d": toy2d,
    "visual": visual_cortex,
    "cortex": whole_cortex,
    "rect2d": rect2d,
    "masked3d": masked3d,
    "paper_toy": paper_toy,
}


def random_unit(n: int, seed: int) -> np.ndarray:
    v = np.random.default_rng(seed).standard_normal(n)
    return v / math.sqrt(float(v @ v))


def smooth_unit(grid: Grid, seed: int, width: float = 0.25) -> np.ndarray:
    """Unit vector of a smooth bump on the grid (a Gaussian of ``width`` in unit
    coordinates around a random active voxel), shaped like the ALS factors of a
    greedy solve: their sub-systems are the ill-conditioned ones."""
    rng = np.random.default_rng(seed)
    c = grid.unit_coords()
    ctr = c[rng.integers(len(c))]
    v = np.exp(-((c - ctr) ** 2).sum(axis=1) / (2.0 * width * width))
    return v / math.sqrt(float(v @ v))
