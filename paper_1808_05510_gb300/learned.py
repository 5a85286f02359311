"""Training and evaluation of the learned preconditioner for the ALS sub-problems.

The network (``conreg.ConvNet``, kernels in ``csrc/cr_net.cu``) maps the
Jacobi-scaled residual of a u-side system (Eq. ALS_linsys) to a correction:
the solver's flexible CG uses z = D^-1 r + s net(D^-1 r / s, mask).  Training
pairs come from the solver itself: at several ranks of a greedy run the ALS
start vector v and the right side R_j v (plus smooth random right sides) are
taken, and the exact correction e = A_hat^-1 r is computed by the library's
PCG to a tight tolerance.  The target is (e - D^-1 r) / s, the part of the
inverse that Jacobi misses.  Training runs the library's own forward, backward
and Adam kernels on the GPU.
"""
from __future__ import annotations

import dataclasses
from typing import List

import numpy as np

from . import conreg
from .synth import Problem


@dataclasses.dataclass
class Pair:
    x: np.ndarray  # (2, D, H, W) float32
    t: np.ndarray  # (D, H, W) float32


def box_mask(grid) -> np.ndarray:
    m = np.asarray(grid.mask, dtype=bool)
    while m.ndim < 3:
        m = m[..., None]
    return m


def jacobi_diag(p: Problem, v: np.ndarray) -> np.ndarray:
    """Diagonal of A_hat (Eq. ALS_linsys) for unit v: lam((L_y^2)_ii + 2c (L_y)_ii + d) + omega_i."""
    Ly = p.Ly.to_dense() if p.ny <= 2000 else None
    Lx_v = _csr_mul(p.Lx, v)
    c = float(v @ Lx_v)
    d = float(Lx_v @ Lx_v)
    diag = np.zeros(p.ny)
    l2 = np.zeros(p.ny)
    for i in range(p.ny):
        for q in range(p.Ly.rowptr[i], p.Ly.rowptr[i + 1]):
            val = p.Ly.val[q]
            l2[i] += val * val
            if p.Ly.col[q] == i:
                diag[i] += val
    xi = p.X.T @ v
    omega = p.Omega.astype(np.float64) @ (xi * xi)
    del Ly
    return p.lam * (l2 + 2.0 * c * diag + d) + omega


def _csr_mul(L, x):
    y = np.zeros(L.n)
    for i in range(L.n):
        s = 0.0
        for q in range(L.rowptr[i], L.rowptr[i + 1]):
            s += L.val[q] * x[L.col[q]]
        y[i] = s
    return y


def _to_box(mask3: np.ndarray, vec: np.ndarray) -> np.ndarray:
    out = np.zeros(mask3.shape, dtype=np.float32)
    out[mask3] = vec
    return out


def smooth_field(p: Problem, rng: np.random.Generator, bumps: int = 6) -> np.ndarray:
    c = p.grid_y.unit_coords()
    f = np.zeros(p.ny)
    for _ in range(bumps):
        ctr = c[rng.integers(len(c))]
        w = rng.uniform(0.05, 0.3)
        f += rng.standard_normal() * np.exp(-((c - ctr) ** 2).sum(1) / (2 * w * w))
    return f


def make_pairs(p: Problem, ranks: List[int], n_random: int = 4, seed: int = 0, tol: float = 1e-9) -> List[Pair]:
    """(input, target) pairs from the u-side systems the greedy solver meets at the given ranks."""
    rng = np.random.default_rng(seed)
    mask3 = box_mask(p.grid_y)
    pairs: List[Pair] = []
    with conreg.ConReg.from_problem(p, r_cap=max(max(ranks), 1), pcg_tol=tol, pcg_maxit=100000) as g:
        done = 0
        for j in sorted(ranks):
            if j > done:
                g.cr_solve(j, 0.0, 0.0)
                done = g.cr_get_rank()
            v = g.cr_apply_residual(np.ones(p.ny), trans=True)
            v /= np.linalg.norm(v)
            Dg = jacobi_diag(p, v)
            rhss = [g.cr_apply_residual(v)] + [smooth_field(p, rng) for _ in range(n_random)]
            for r in rhss:
                e, _ = g.cr_solve_u(v, r)
                jr = r / Dg
                s = float(np.linalg.norm(jr))
                if s == 0.0:
                    continue
                x = np.stack([_to_box(mask3, jr / s), mask3.astype(np.float32)])
                pairs.append(Pair(x.transpose(0, 1, 2, 3).astype(np.float32), _to_box(mask3, (e - jr) / s)))
    return pairs


def train(net: "conreg.ConvNet", pairs: List[Pair], steps: int = 300, lr: float = 2e-3, batch: int = 4,
          seed: int = 0, log_every: int = 0):
    """Adam on the relative masked error; returns the loss history."""
    import torch

    rng = np.random.default_rng(seed)
    dev = torch.device("cuda", torch.cuda.current_device())
    X = torch.tensor(np.stack([q.x for q in pairs]), device=dev)
    T = torch.tensor(np.stack([q.t for q in pairs]), device=dev)
    mask = (X[0, 1] > 0).to(torch.uint8).contiguous()
    hist = []
    for it in range(steps):
        idx = torch.tensor(rng.choice(len(pairs), size=min(batch, len(pairs)), replace=False), device=dev)
        loss = net.train_step(X[idx], T[idx], mask, lr)
        hist.append(loss)
        if log_every and it % log_every == 0:
            print(f"step {it} loss {loss:.4f}", flush=True)
    return hist


def compare_iterations(p: Problem, net: "conreg.ConvNet", ranks: List[int], tol: float = 1e-8):
    """Iterations of Jacobi-PCG and of the learned flexible CG on the same u-side systems."""
    out = []
    with conreg.ConReg.from_problem(p, r_cap=max(max(ranks), 1), pcg_tol=tol, pcg_maxit=100000) as gj, \
            conreg.ConReg.from_problem(p, r_cap=max(max(ranks), 1), pcg_tol=tol, pcg_maxit=100000,
                                       precond=conreg.CR_PRECOND_LEARNED) as gl:
        gl.cr_set_voxel_grid(0, p.grid_y.mask)
        gl.cr_set_voxel_grid(1, p.grid_x.mask)
        gl.cr_set_preconditioner(net)
        done = 0
        for j in sorted(ranks):
            if j > done:
                gj.cr_solve(j, 0.0, 0.0)
                done = gj.cr_get_rank()
            U, Z, V = gj.cr_get_factors()
            if U.shape[1]:
                gl.cr_set_factors(U, Z, V)
            v = gj.cr_apply_residual(np.ones(p.ny), trans=True)
            v /= np.linalg.norm(v)
            r = gj.cr_apply_residual(v)
            ej, itj = gj.cr_solve_u(v, r)
            el, itl = gl.cr_solve_u(v, r)
            out.append({"rank": j, "iters_jacobi": itj, "iters_learned": itl,
                        "rel_diff": float(np.linalg.norm(el - ej) / np.linalg.norm(ej))})
    return out
