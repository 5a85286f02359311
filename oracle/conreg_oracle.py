"""CPU float64 oracle for the greedy low-rank connectome regression.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import or call this
module: only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` use it.  It shares no code with the CUDA library; it is a plain,
slow restatement of the paper (Kuerschner, Dolgov, Harris, Benner,
"Greedy low-rank algorithm for spatial connectome regression"):

* the objective, Eq. (obj_fun), and its normal equations, Eqs. (linear_system),
  (system_matrix), (multitermSylv) of Sec. 2.1;
* the ALS half-steps, Eqs. (ALS_linsys), (ALS_linsys_v) of Sec. 2.3;
* the Galerkin equation, Eq. (Proj_Sylv), solved by matrix-valued CG with the
  previous Z as initial guess (Sec. 2.3) or, for small rank, by the assembled
  Kronecker matrix;
* Algorithm 1 (greedy rank-1 method with Galerkin projection).

Library primitives (dense/sparse matrix products, Cholesky) serve as single
steps; nothing is blocked or fused beyond what the equations state.  Where the
paper is silent the oracle takes these readings:

* ALS start vector: ``v0 = R_j^T 1 / ||R_j^T 1||`` (a seeded Gaussian if that
  norm vanishes); at least one ALS sweep, at most ``als_max_iter``; the sweep
  loop stops when ``delta = | ||u_hat|| / ||v_hat|| - 1 | <= als_delta``.
* ``orth`` is classical Gram-Schmidt applied twice; a column whose norm after
  projection is below ``1e-12`` of its norm before is rejected (rank deficient).
* Galerkin CG stops when ``||U^T D V - K(Z)||_F <= tol * ||U^T D V||_F``.
* The sub-systems with A_hat / B_hat are solved exactly: dense Cholesky for
  n <= ``dense_max``, otherwise Jacobi-preconditioned CG to ``cg_tol``.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Callable, List, Optional

import numpy as np
import scipy.sparse as sp

__all__ = ["Oracle", "GreedyResult", "cholesky_solve", "cg"]


# ----------------------------------------------------------------------------
# Small dense / iterative linear algebra used as single steps
# ----------------------------------------------------------------------------

def cholesky_solve(A: np.ndarray, b: np.ndarray) -> np.ndarray:
    """Solve an SPD system through numpy's Cholesky factor."""
    Lc = np.linalg.cholesky(A)
    y = np.linalg.solve(Lc, b)
    return np.linalg.solve(Lc.T, y)


def cg(apply: Callable[[np.ndarray], np.ndarray], b: np.ndarray, x0: Optional[np.ndarray] = None,
       tol: float = 1e-14, maxit: int = 100000, precond: Optional[np.ndarray] = None,
       inner: Callable[[np.ndarray, np.ndarray], float] = lambda a, c: float(np.vdot(a, c))):
    """Textbook (preconditioned) conjugate gradients with the relative residual
    stopping test ``||b - A x|| <= tol ||b||``.  Works for vectors and, with the
    Frobenius inner product, for matrices.  Returns (x, iterations, relres)."""
    x = np.zeros_like(b) if x0 is None else x0.copy()
    r = b - apply(x)
    bn = math.sqrt(inner(b, b))
    if bn == 0.0:
        return np.zeros_like(b), 0, 0.0
    z = r * precond if precond is not None else r
    p = z.copy()
    rz = inner(r, z)
    it = 0
    rn = math.sqrt(inner(r, r))
    while rn > tol * bn and it < maxit:
        q = apply(p)
        alpha = rz / inner(p, q)
        x = x + alpha * p
        r = r - alpha * q
        z = r * precond if precond is not None else r
        rz_new = inner(r, z)
        p = z + (rz_new / rz) * p
        rz = rz_new
        rn = math.sqrt(inner(r, r))
        it += 1
    return x, it, rn / bn


# ----------------------------------------------------------------------------
# The problem and its operators
# ----------------------------------------------------------------------------

@dataclasses.dataclass
class GreedyStep:
    j: int
    sweeps: int
    delta: float
    unorm: float
    vnorm: float
    galerkin_iters: int
    dW: float
    relres: float
    J: float


@dataclasses.dataclass
class GreedyResult:
    U: np.ndarray
    Z: np.ndarray
    V: np.ndarray
    steps: List[GreedyStep]
    stop: str

    @property
    def W(self) -> np.ndarray:
        return self.U @ self.Z @ self.V.T


class Oracle:
    """Plain float64 statement of the problem

        min_W 1/2 ||(W X - Y) o Omega||_F^2 + lambda/2 ||L_y W + W L_x^T||_F^2   (Eq. obj_fun)

    built from CSR Laplacians and dense ``X`` (nx x m), ``Y`` (ny x m),
    ``Omega`` (ny x m, 1 = observed)."""

    def __init__(self, Lx_csr, Ly_csr, X, Y, Omega, lam, dense_max: int = 2000, cg_tol: float = 1e-14):
        self.Lx = sp.csr_matrix((Lx_csr.val, Lx_csr.col, Lx_csr.rowptr), shape=(Lx_csr.n, Lx_csr.n))
        self.Ly = sp.csr_matrix((Ly_csr.val, Ly_csr.col, Ly_csr.rowptr), shape=(Ly_csr.n, Ly_csr.n))
        self.X = np.asarray(X, dtype=np.float64)
        self.Y = np.asarray(Y, dtype=np.float64)
        self.Om = np.asarray(Omega, dtype=np.float64)
        self.lam = float(lam)
        self.nx, self.m = self.X.shape
        self.ny = self.Y.shape[0]
        self.dense_max = dense_max
        self.cg_tol = cg_tol
        self.Lx2 = (self.Lx @ self.Lx).tocsr()
        self.Ly2 = (self.Ly @ self.Ly).tocsr()

    @classmethod
    def from_problem(cls, p, **kw) -> "Oracle":
        return cls(p.Lx, p.Ly, p.X, p.Y, p.Omega, p.lam, **kw)

    # --- Sec. 2.1 ------------------------------------------------------------
    def D(self) -> np.ndarray:
        """Right-hand side D = (Omega o Y) X^T (Eq. multitermSylv)."""
        return (self.Om * self.Y) @ self.X.T

    def B_op(self, W: np.ndarray) -> np.ndarray:
        """Smoothing operator B(W) = W L_x^2 + 2 L_y W L_x + L_y^2 W (Eq. multitermSylv)."""
        return (self.Lx2.T @ W.T).T + 2.0 * (self.Lx.T @ (self.Ly @ W).T).T + self.Ly2 @ W

    def C_op(self, W: np.ndarray) -> np.ndarray:
        """Data operator C(W) = sum_alpha diag(Omega_alpha) W X_alpha X_alpha^T (Eq. multitermSylv)."""
        out = np.zeros_like(W)
        for a in range(self.m):
            xa = self.X[:, a]
            out += np.outer(self.Om[:, a] * (W @ xa), xa)
        return out

    def A_op(self, W: np.ndarray) -> np.ndarray:
        """A(W) = lambda B(W) + C(W) (Eq. multitermSylv)."""
        return self.lam * self.B_op(W) + self.C_op(W)

    def A_dense(self) -> np.ndarray:
        """The (ny nx) x (ny nx) matrix of Eq. (system_matrix), Kronecker products
        acting on vec(W) (columns stacked)."""
        Iy = np.eye(self.ny)
        Ix = np.eye(self.nx)
        Lx = self.Lx.toarray()
        Ly = self.Ly.toarray()
        A = self.lam * (np.kron(Lx @ Lx, Iy) + 2.0 * np.kron(Lx, Ly) + np.kron(Ix, Ly @ Ly))
        for a in range(self.m):
            xa = self.X[:, a]
            A += np.kron(np.outer(xa, xa), np.diag(self.Om[:, a]))
        return A

    def J(self, W: np.ndarray) -> float:
        """Objective of Eq. (obj_fun)."""
        loss = 0.5 * np.sum(((W @ self.X - self.Y) * self.Om) ** 2)
        S = self.Ly @ W + (self.Lx @ W.T).T  # L_y W + W L_x^T
        return float(loss + 0.5 * self.lam * np.sum(S * S))

    def solve_full(self, tol: float = 1e-14) -> np.ndarray:
        """W* of Eq. (linear_system): dense Cholesky of A when small, else CG on A."""
        N = self.ny * self.nx
        rhs = self.D()
        if N <= 4000:
            w = cholesky_solve(self.A_dense(), rhs.reshape(-1, order="F"))
            return w.reshape(self.ny, self.nx, order="F")
        W, _, _ = cg(self.A_op, rhs, tol=tol, maxit=200000,
                     inner=lambda a, c: float(np.sum(a * c)))
        return W

    # --- residual products R_j v and R_j^T u (matrix-free, W = U Z V^T) -----
    def R_dense(self, U, Z, V) -> np.ndarray:
        """R = D - A(U Z V^T), formed densely (Algorithm 1, residual update)."""
        return self.D() - self.A_op(U @ Z @ V.T)

    def _AW_times(self, U, Z, V, v: np.ndarray) -> np.ndarray:
        """A(W) v for W = U Z V^T, each product of Eq. (multitermSylv) evaluated
        right to left: lambda (W L_x^2 v + 2 L_y W L_x v + L_y^2 W v)
        + ((W X) o Omega) X^T v."""
        if U.shape[1] == 0:
            return np.zeros(self.ny)
        W_ = lambda w: U @ (Z @ (V.T @ w))
        out = self.lam * (W_(self.Lx2 @ v) + 2.0 * (self.Ly @ W_(self.Lx @ v)) + self.Ly2 @ W_(v))
        WX = U @ (Z @ (V.T @ self.X))
        return out + (WX * self.Om) @ (self.X.T @ v)

    def _AWt_times(self, U, Z, V, u: np.ndarray) -> np.ndarray:
        """A(W)^T u for W = U Z V^T (transpose of each term of Eq. multitermSylv)."""
        if U.shape[1] == 0:
            return np.zeros(self.nx)
        Wt = lambda w: V @ (Z.T @ (U.T @ w))
        out = self.lam * (self.Lx2 @ Wt(u) + 2.0 * (self.Lx @ Wt(self.Ly @ u)) + Wt(self.Ly2 @ u))
        WX = U @ (Z @ (V.T @ self.X))
        return out + self.X @ ((WX * self.Om).T @ u)

    def R_times(self, U, Z, V, v: np.ndarray) -> np.ndarray:
        """R_j v with R_j = D - A(U Z V^T) (right side of Eq. ALS_linsys);
        D v = (Omega o Y)(X^T v)."""
        return (self.Om * self.Y) @ (self.X.T @ v) - self._AW_times(U, Z, V, v)

    def Rt_times(self, U, Z, V, u: np.ndarray) -> np.ndarray:
        """R_j^T u (right side of Eq. ALS_linsys_v); D^T u = X ((Omega o Y)^T u)."""
        return self.X @ ((self.Om * self.Y).T @ u) - self._AWt_times(U, Z, V, u)

    # --- Sec. 2.3: ALS ---------------------------------------------------------
    def A_hat(self, v: np.ndarray):
        """A_hat of Eq. (ALS_linsys) for unit v, as a sparse matrix."""
        cLx2 = float(v @ (self.Lx2 @ v))
        cLx = float(v @ (self.Lx @ v))
        w = (self.X.T @ v) ** 2  # v^T X_a X_a^T v
        diag = self.Om @ w
        Iy = sp.identity(self.ny, format="csr")
        return (self.lam * (cLx2 * Iy + 2.0 * cLx * self.Ly + self.Ly2) + sp.diags(diag)).tocsr()

    def B_hat(self, u: np.ndarray) -> np.ndarray:
        """B_hat of Eq. (ALS_linsys_v) for unit u, dense (sparse part + rank-m part)."""
        cLy = float(u @ (self.Ly @ u))
        cLy2 = float(u @ (self.Ly2 @ u))
        s = self.Om.T @ (u * u)  # u^T diag(Omega_a) u
        Ix = sp.identity(self.nx, format="csr")
        Bs = self.lam * (self.Lx2 + 2.0 * cLy * self.Lx + cLy2 * Ix)
        return Bs, s

    def _solve_sparse_plus(self, S, s_lowrank, rhs, x0=None):
        n = rhs.shape[0]
        if s_lowrank is None:
            apply = lambda p: S @ p
            diag = S.diagonal()
        else:
            Xs = self.X
            apply = lambda p: S @ p + Xs @ (s_lowrank * (Xs.T @ p))
            diag = S.diagonal() + (Xs * Xs) @ s_lowrank
        if n <= self.dense_max:
            M = S.toarray()
            if s_lowrank is not None:
                M = M + (self.X * s_lowrank) @ self.X.T
            return cholesky_solve(M, rhs), 0
        x, it, _ = cg(apply, rhs, x0=x0, tol=self.cg_tol, maxit=50 * n, precond=1.0 / diag)
        return x, it

    def solve_u(self, v, rhs, x0=None):
        """u_hat = A_hat^{-1} rhs (Eq. ALS_linsys)."""
        return self._solve_sparse_plus(self.A_hat(v), None, rhs, x0)[0]

    def solve_v(self, u, rhs, x0=None):
        """v_hat = B_hat^{-1} rhs (Eq. ALS_linsys_v)."""
        S, s = self.B_hat(u)
        return self._solve_sparse_plus(S, s, rhs, x0)[0]

    # --- orth ----------------------------------------------------------------
    @staticmethod
    def orth_append(Q: np.ndarray, u: np.ndarray, rej: float = 1e-12):
        """Append u to the orthonormal columns of Q by classical Gram-Schmidt
        applied twice; returns (new Q, accepted)."""
        nrm0 = float(np.linalg.norm(u))
        w = u.copy()
        for _ in range(2):
            if Q.shape[1]:
                w = w - Q @ (Q.T @ w)
        nrm = float(np.linalg.norm(w))
        if nrm0 == 0.0 or nrm < rej * nrm0:
            return Q, False
        return np.column_stack([Q, w / nrm]), True

    # --- Galerkin (Eq. Proj_Sylv) ----------------------------------------------
    def projected(self, U, V):
        """Coefficient matrices of Eq. (Proj_Sylv)."""
        A1 = U.T @ (self.Ly @ U)
        A2 = U.T @ (self.Ly2 @ U)
        B1 = V.T @ (self.Lx @ V)
        B2 = V.T @ (self.Lx2 @ V)
        G = [U.T @ (self.Om[:, a][:, None] * U) for a in range(self.m)]
        Hs = [np.outer(V.T @ self.X[:, a], V.T @ self.X[:, a]) for a in range(self.m)]
        F = (U.T @ (self.Om * self.Y)) @ (self.X.T @ V)  # U^T D V
        return A1, A2, B1, B2, G, Hs, F

    def K_apply(self, Z, A1, A2, B1, B2, G, Hs):
        """Left side of Eq. (Proj_Sylv) applied to Z."""
        out = self.lam * (Z @ B2 + 2.0 * A1 @ Z @ B1 + A2 @ Z)
        for Ga, Ha in zip(G, Hs):
            out = out + Ga @ Z @ Ha
        return out

    def K_dense(self, A1, A2, B1, B2, G, Hs):
        """Eq. (Proj_Sylv) as a j^2 x j^2 matrix on vec(Z)."""
        j = A1.shape[0]
        I = np.eye(j)
        K = self.lam * (np.kron(B2.T, I) + 2.0 * np.kron(B1.T, A1) + np.kron(I, A2))
        for Ga, Ha in zip(G, Hs):
            K += np.kron(Ha.T, Ga)
        return K

    def galerkin(self, U, V, Z0=None, tol=1e-14, direct_max_j: int = 60, maxit=None):
        """Solve Eq. (Proj_Sylv) for Z: Kronecker + Cholesky for j <= direct_max_j
        ("exact"), otherwise matrix CG from Z0 to ``tol``.  Returns (Z, iters)."""
        A1, A2, B1, B2, G, Hs, F = self.projected(U, V)
        j = U.shape[1]
        if j <= direct_max_j and tol <= 1e-13:
            z = cholesky_solve(self.K_dense(A1, A2, B1, B2, G, Hs), F.reshape(-1, order="F"))
            return z.reshape(j, j, order="F"), 0
        Z, it, _ = cg(lambda Zm: self.K_apply(Zm, A1, A2, B1, B2, G, Hs), F, x0=Z0, tol=tol,
                      maxit=maxit or 10 * j * j + 100, inner=lambda a, c: float(np.sum(a * c)))
        return Z, it

    # --- held-out scoring -------------------------------------------------------
    @staticmethod
    def cv_error(U, Z, V, Xt, Yt, Omt):
        """Twice the data term of Eq. (obj_fun) on held-out injections, for
        W = U Z V^T: (sum |(W X_t - Y_t) o Omega_t|^2, sum |Y_t o Omega_t|^2).
        The second value is the first at W = 0.  (The paper fixes lambda-bar
        by hand, Sec. 1.1; scoring held-out injections is the reading used for
        the lambda x fold sweep.)"""
        Om = np.asarray(Omt, dtype=np.float64)
        W = np.asarray(U) @ np.asarray(Z) @ np.asarray(V).T
        E = (W @ np.asarray(Xt) - np.asarray(Yt)) * Om
        Y0 = np.asarray(Yt) * Om
        return float(np.sum(E * E)), float(np.sum(Y0 * Y0))

    # --- Algorithm 1 -------------------------------------------------------------
    def greedy(self, r_max: int, tau: float = 1e-12, relres_target: float = 0.0, als_delta: float = 0.1,
               als_max_iter: int = 10, als_sweeps: Optional[int] = None, galerkin_tol: Optional[float] = None,
               seed: int = 1808, callback=None, dense_residual: bool = True) -> GreedyResult:
        """Algorithm 1: greedy rank-1 updates by ALS, orthogonalisation, Galerkin
        projection (CG to tau/2 unless ``galerkin_tol`` is given), residual, and the
        relative-change stopping test ``dW <= tau``.  ``als_sweeps`` fixes the number
        of ALS sweeps (deterministic comparison mode)."""
        ny, nx = self.ny, self.nx
        U = np.zeros((ny, 0))
        V = np.zeros((nx, 0))
        Z = np.zeros((0, 0))
        Dn = float(np.linalg.norm(self.D()))
        steps: List[GreedyStep] = []
        gtol = tau / 2.0 if galerkin_tol is None else galerkin_tol
        stop = "r_max"
        u_hat = None
        for j in range(r_max):
            # ALS start vector (reading: R_j^T 1, normalised)
            v = self.Rt_times(U, Z, V, np.ones(ny))
            vn = float(np.linalg.norm(v))
            if vn <= 1e-300 * max(Dn, 1e-300):
                g = np.random.default_rng(seed + j).standard_normal(nx)
                v = g / np.linalg.norm(g)
            else:
                v = v / vn
            sweeps = 0
            delta = math.inf
            while True:
                rhs_u = self.R_times(U, Z, V, v)
                u_hat = self.solve_u(v, rhs_u)
                un = float(np.linalg.norm(u_hat))
                u = u_hat / un
                rhs_v = self.Rt_times(U, Z, V, u)
                v_hat = self.solve_v(u, rhs_v)
                vn = float(np.linalg.norm(v_hat))
                v = v_hat / vn
                delta = abs(un / vn - 1.0)
                sweeps += 1
                if als_sweeps is not None:
                    if sweeps >= als_sweeps:
                        break
                elif delta <= als_delta or sweeps >= als_max_iter:
                    break
            U_new, oku = self.orth_append(U, u)
            V_new, okv = self.orth_append(V, v)
            if not (oku and okv):
                stop = "rank_deficient"
                break
            W_prev = U @ Z @ V.T if U.shape[1] else None
            Z0 = np.zeros((j + 1, j + 1))
            Z0[:j, :j] = Z
            U, V = U_new, V_new
            Z, git = self.galerkin(U, V, Z0, tol=gtol)
            W = U @ Z @ V.T
            dW = float(np.linalg.norm(W - (W_prev if W_prev is not None else 0.0)) / np.linalg.norm(W))
            relres = float(np.linalg.norm(self.D() - self.A_op(W)) / Dn) if dense_residual else float("nan")
            st = GreedyStep(j + 1, sweeps, delta, un, vn, git, dW, relres, self.J(W))
            steps.append(st)
            if callback is not None:
                callback(st, U, Z, V)
            if dW <= tau:
                stop = "dW"
                break
            if relres_target > 0.0 and relres <= relres_target:
                stop = "relres"
                break
        return GreedyResult(U, Z, V, steps, stop)
