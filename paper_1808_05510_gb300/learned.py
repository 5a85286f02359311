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
    return p.lam * (l2 + 2.0 * c * diag + d) + omega


def jacobi_diag_v(p: Problem, u: np.ndarray) -> np.ndarray:
    """Diagonal of B_hat (Eq. ALS_linsys_v) for unit u: lam((L_x^2)_kk + 2c' (L_x)_kk + d') + sum_a s_a X_ka^2."""
    Ly_u = _csr_mul(p.Ly, u)
    c = float(u @ Ly_u)
    d = float(Ly_u @ Ly_u)
    diag = np.zeros(p.nx)
    l2 = np.zeros(p.nx)
    for i in range(p.nx):
        for q in range(p.Lx.rowptr[i], p.Lx.rowptr[i + 1]):
            val = p.Lx.val[q]
            l2[i] += val * val
            if p.Lx.col[q] == i:
                diag[i] += val
    s = p.Omega.astype(np.float64).T @ (u * u)
    return p.lam * (l2 + 2.0 * c * diag + d) + (p.X * p.X) @ s


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


def smooth_field(p: Problem, rng: np.random.Generator, bumps: int = 6, side: int = 0) -> np.ndarray:
    """Sum of random Gaussian bumps on the y grid (side 0) or the x grid (side 1)."""
    c = (p.grid_y if side == 0 else p.grid_x).unit_coords()
    f = np.zeros(len(c))
    for _ in range(bumps):
        ctr = c[rng.integers(len(c))]
        w = rng.uniform(0.05, 0.3)
        f += rng.standard_normal() * np.exp(-((c - ctr) ** 2).sum(1) / (2 * w * w))
    return f


def make_pairs(p: Problem, ranks: List[int], n_random: int = 4, seed: int = 0, tol: float = 1e-9,
               sides=(0, 1)) -> List[Pair]:
    """(input, target) pairs from the sub-systems the greedy solver meets at the
    given ranks: u side (Eq. ALS_linsys) for the ALS start vector v, v side
    (Eq. ALS_linsys_v) for u = u_hat / |u_hat|, each with its right side from the
    residual plus n_random smooth random right sides."""
    rng = np.random.default_rng(seed)
    masks = [box_mask(p.grid_y), box_mask(p.grid_x)]
    pairs: List[Pair] = []

    def add(side, r, e, Dg):
        jr = r / Dg
        s = float(np.linalg.norm(jr))
        if s == 0.0:
            return
        m3 = masks[side]
        x = np.stack([_to_box(m3, jr / s), m3.astype(np.float32)])
        pairs.append(Pair(x.astype(np.float32), _to_box(m3, (e - jr) / s)))

    with conreg.ConReg.from_problem(p, r_cap=max(max(ranks), 1), pcg_tol=tol, pcg_maxit=100000) as g:
        done = 0
        for j in sorted(ranks):
            if j > done:
                g.cr_solve(j, 0.0, 0.0)
                done = g.cr_get_rank()
            v = g.cr_apply_residual(np.ones(p.ny), trans=True)
            v /= np.linalg.norm(v)
            Du = jacobi_diag(p, v)
            ru = g.cr_apply_residual(v)
            eu, _ = g.cr_solve_u(v, ru)
            if 0 in sides:
                add(0, ru, eu, Du)
                for _ in range(n_random):
                    r = smooth_field(p, rng)
                    add(0, r, g.cr_solve_u(v, r)[0], Du)
            if 1 in sides:
                u = eu / np.linalg.norm(eu)
                Dv = jacobi_diag_v(p, u)
                rv = g.cr_apply_residual(u, trans=True)
                add(1, rv, g.cr_solve_v(u, rv)[0], Dv)
                for _ in range(n_random):
                    r = smooth_field(p, rng, side=1)
                    add(1, r, g.cr_solve_v(u, r)[0], Dv)
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


def compare_iterations(p: Problem, net: "conreg.ConvNet", ranks: List[int], tol: float = 1e-8, sides=(0,)):
    """Iterations of Jacobi-PCG and of the learned flexible CG on the same sub-systems.

    The learned problem's first solve on each side is its Jacobi judge run
    (cr_set_preconditioner), so one calibration solve per side precedes the
    measured ones; the judge counts iterations (what the network changes)."""
    out = []
    with conreg.ConReg.from_problem(p, r_cap=max(max(ranks), 1), pcg_tol=tol, pcg_maxit=100000) as gj, \
            conreg.ConReg.from_problem(p, r_cap=max(max(ranks), 1), pcg_tol=tol, pcg_maxit=100000,
                                       precond=conreg.CR_PRECOND_LEARNED, learned_judge=1) as gl:
        gl.cr_set_voxel_grid(0, p.grid_y.mask)
        gl.cr_set_voxel_grid(1, p.grid_x.mask)
        gl.cr_set_preconditioner(net)
        done = 0
        calibrated = False
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
            if not calibrated:
                gl.cr_solve_u(v, r)
                gl.cr_solve_v(ej / np.linalg.norm(ej), gj.cr_apply_residual(ej / np.linalg.norm(ej), trans=True))
                calibrated = True
            if 0 in sides:
                el, itl = gl.cr_solve_u(v, r)
                out.append({"rank": j, "side": "u", "iters_jacobi": itj, "iters_learned": itl,
                            "rel_diff": float(np.linalg.norm(el - ej) / np.linalg.norm(ej))})
            if 1 in sides:
                u = ej / np.linalg.norm(ej)
                rv = gj.cr_apply_residual(u, trans=True)
                fj, itj2 = gj.cr_solve_v(u, rv)
                fl, itl2 = gl.cr_solve_v(u, rv)
                out.append({"rank": j, "side": "v", "iters_jacobi": itj2, "iters_learned": itl2,
                            "rel_diff": float(np.linalg.norm(fl - fj) / np.linalg.norm(fj))})
    return out


def train_for(problems: List[Problem], ranks: List[int], steps: int = 300, n_random: int = 3, batch: int = 8,
              lr: float = 2e-3, seed: int = 1):
    """Pairs from every problem (both sides) and a trained network on their common box."""
    pairs = []
    for k, p in enumerate(problems):
        pairs += make_pairs(p, ranks, n_random=n_random, seed=seed + k)
    shape = pairs[0].t.shape
    net = conreg.ConvNet(shape, batch_cap=batch, seed=seed)
    hist = train(net, pairs, steps=steps, lr=lr, batch=batch, seed=seed)
    return net, hist, len(pairs)
