"""The multigrid hierarchy builder (csrc/cr_mg_host.h), built on the CPU with g++
and checked against its definitions with scipy: every row in exactly one
connected aggregate; P = (I - omega D^-1 L) P0; Galerkin coarse matrices
L_{l+1} = P^T L_l P and M_{l+1} = P^T M_l P; constants exact on every level
(L_l P_l 1 = 0); and, as a preconditioner for the sub-problem operators of
Sec. 2.3, two V-cycles of L + sigma I beating Jacobi by a wide margin."""
import ctypes as C
import math
import os
import shutil
import subprocess

import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.csgraph as csg

from paper_1808_05510_gb300 import synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER_DIR = os.path.join(ROOT, "paper_1808_05510_gb300", "csrc")

WRAPPER = r"""
#include "cr_mg_host.h"
static cr_mg::Hierarchy H;
static std::vector<int> AGG0;
extern "C" int t_build(int n, const int* rp, const int* ci, const double* v, int coarse_max) {
  cr_mg::Csr L;
  L.rows = L.cols = n;
  L.rp.assign(rp, rp + n + 1);
  L.ci.assign(ci, ci + rp[n]);
  L.v.assign(v, v + rp[n]);
  H = cr_mg::build(L, coarse_max);
  int na = 0;
  AGG0 = cr_mg::aggregate(L, &na);
  return (int)H.lev.size();
}
static const cr_mg::Csr& pick(int l, int which) {
  const cr_mg::Level& x = H.lev[l];
  return which == 0 ? x.L : which == 1 ? x.M : which == 2 ? x.P : x.R;
}
extern "C" void t_shape(int l, int which, int* out) {
  const cr_mg::Csr& A = pick(l, which);
  out[0] = A.rows; out[1] = A.cols; out[2] = (int)A.nnz();
}
extern "C" void t_copy(int l, int which, int* rp, int* ci, double* v) {
  const cr_mg::Csr& A = pick(l, which);
  std::copy(A.rp.begin(), A.rp.end(), rp);
  std::copy(A.ci.begin(), A.ci.end(), ci);
  std::copy(A.v.begin(), A.v.end(), v);
}
extern "C" void t_agg0(int* out) { std::copy(AGG0.begin(), AGG0.end(), out); }
extern "C" int t_pencil(double* Q, double* mu) {
  std::vector<double> q, w;
  const cr_mg::Level& c = H.lev.back();
  if (!cr_mg::pencil_basis(c.L, c.M, q, w)) return 0;
  std::copy(q.begin(), q.end(), Q);
  std::copy(w.begin(), w.end(), mu);
  return 1;
}
"""


@pytest.fixture(scope="module")
def lib(tmp_path_factory):
    if shutil.which("g++") is None:
        pytest.skip("g++ not available")
    d = tmp_path_factory.mktemp("hostmg")
    src = d / "w.cpp"
    src.write_text(WRAPPER)
    so = d / "libw.so"
    subprocess.run(["g++", "-std=c++17", "-O2", "-shared", "-fPIC", "-I", HEADER_DIR, str(src), "-o", str(so)],
                   check=True)
    return C.CDLL(str(so))


def build(lib, L, coarse_max=64):
    ip = np.ctypeslib.ndpointer(dtype=np.int32, flags="C_CONTIGUOUS")
    dp = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")
    lib.t_build.argtypes = [C.c_int, ip, ip, dp, C.c_int]
    nlev = lib.t_build(L.n, np.ascontiguousarray(L.rowptr, np.int32), np.ascontiguousarray(L.col, np.int32),
                       np.ascontiguousarray(L.val, np.float64), coarse_max)
    levels = []
    for l in range(nlev):
        mats = []
        for which in range(4):
            shp = np.zeros(3, np.int32)
            lib.t_shape(l, which, shp.ctypes.data_as(C.POINTER(C.c_int)))
            r, c, nnz = (int(x) for x in shp)
            rp = np.zeros(r + 1, np.int32)
            ci = np.zeros(max(nnz, 1), np.int32)
            v = np.zeros(max(nnz, 1))
            lib.t_copy(l, which, rp.ctypes.data_as(C.POINTER(C.c_int)), ci.ctypes.data_as(C.POINTER(C.c_int)),
                       v.ctypes.data_as(C.POINTER(C.c_double)))
            mats.append(sp.csr_matrix((v[:nnz], ci[:nnz], rp), shape=(r, c)) if r else None)
        levels.append(dict(zip("LMPR", mats)))
    agg = np.zeros(L.n, np.int32)
    lib.t_agg0(agg.ctypes.data_as(C.POINTER(C.c_int)))
    return levels, agg


def csr(L):
    return sp.csr_matrix((L.val, L.col, L.rowptr), shape=(L.n, L.n))


PROBLEMS = {"chain200": lambda: synth.paper_toy(), "toy2d": lambda: synth.toy2d(), "masked3d": lambda: synth.masked3d()}


@pytest.fixture(scope="module", params=list(PROBLEMS))
def hier(request, lib):
    p = PROBLEMS[request.param]()
    return p, csr(p.Ly), *build(lib, p.Ly)


def test_aggregates_partition_rows_into_connected_sets(hier):
    _, L, levels, agg = hier
    n = L.shape[0]
    na = levels[1]["L"].shape[0]
    assert agg.min() == 0 and agg.max() == na - 1 and na < n
    assert np.array_equal(np.unique(agg), np.arange(na))
    adj = (L - sp.diags(L.diagonal())).tocsr()
    adj.data[:] = 1.0
    for a in range(na):
        idx = np.flatnonzero(agg == a)
        ncomp, _ = csg.connected_components(adj[idx][:, idx], directed=False)
        assert ncomp == 1


def test_prolongation_is_smoothed_aggregation(hier):
    _, L, levels, agg = hier
    n, na = L.shape[0], levels[1]["L"].shape[0]
    P0 = sp.csr_matrix((np.ones(n), (np.arange(n), agg)), shape=(n, na))
    D = L.diagonal()
    P = (sp.identity(n) - (2.0 / 3.0) * sp.diags(1.0 / D) @ L) @ P0
    assert abs(levels[0]["P"] - P).max() < 1e-15
    assert abs(levels[0]["R"] - P.T).max() < 1e-15


def test_galerkin_coarse_matrices(hier):
    _, L, levels, _ = hier
    for f, c in zip(levels[:-1], levels[1:]):
        P = f["P"]
        scale = abs(c["L"]).max()
        assert abs(c["L"] - P.T @ f["L"] @ P).max() <= 1e-13 * scale
        assert abs(c["M"] - P.T @ f["M"] @ P).max() <= 1e-13 * abs(c["M"]).max()
        assert abs(c["L"] - c["L"].T).max() <= 1e-13 * scale
        # constants stay exact: P 1 = 1 and the coarse Laplacian annihilates 1
        assert np.abs(P @ np.ones(P.shape[1]) - 1.0).max() < 1e-13
        assert np.abs(c["L"] @ np.ones(c["L"].shape[0])).max() <= 1e-12 * scale
    assert levels[-1]["L"].shape[0] <= 64
    assert np.linalg.eigvalsh(levels[-1]["M"].toarray()).min() > 0.0


def vcycle(levels, sigma, r, l=0):
    lev = levels[l]
    A = (lev["L"] + sigma * lev["M"]).tocsr()
    if lev["P"] is None:
        return np.linalg.solve(A.toarray(), r)
    d = A.diagonal()
    x = (2.0 / 3.0) * r / d
    x = x + (2.0 / 3.0) * (r - A @ x) / d
    x = x + lev["P"] @ vcycle(levels, sigma, lev["R"] @ (r - A @ x), l + 1)
    for _ in range(2):
        x = x + (2.0 / 3.0) * (r - A @ x) / d
    return x


def pcg_iters(A, b, prec, tol=1e-10):
    x = np.zeros_like(b)
    r = b.copy()
    z = prec(r)
    p = z.copy()
    rz = r @ z
    it = 0
    while np.linalg.norm(r) > tol * np.linalg.norm(b) and it < 20000:
        q = A @ p
        a = rz / (p @ q)
        x += a * p
        r -= a * q
        z = prec(r)
        rz2 = r @ z
        p = z + (rz2 / rz) * p
        rz = rz2
        it += 1
    return it


def test_two_vcycles_precondition_the_squared_operator(hier):
    """lam [(L + cI)^2 + e I] + diag(w) with a smooth ALS factor's small shift
    (the ill-conditioned case): two V-cycles of L + sigma I, sigma^2 = c^2 + e
    + mean(w)/lam, take a fraction of Jacobi's iterations."""
    p, L, levels, _ = hier
    n = L.shape[0]
    lam, c, e = 100.0, 0.01, 1e-4
    w = np.random.default_rng(5).uniform(0.5, 1.0, n)
    Lc = L + c * sp.identity(n)
    A = (lam * (Lc @ Lc + e * sp.identity(n)) + sp.diags(w)).tocsr()
    b = np.random.default_rng(6).standard_normal(n)
    sigma = math.sqrt(c * c + e + w.mean() / lam)
    it_mg = pcg_iters(A, b, lambda r: vcycle(levels, sigma, vcycle(levels, sigma, r)) / lam)
    it_j = pcg_iters(A, b, lambda r: r / A.diagonal())
    assert it_mg <= 30 and 4 * it_mg < it_j, (it_mg, it_j)


def test_coarsest_pencil_basis_inverts_every_shift(lib, hier):
    """(L_c + sigma M_c)^-1 = Q diag(1 / (mu + sigma)) Q^T with Q^T M_c Q = I."""
    _, _, levels, _ = hier
    Lc, Mc = levels[-1]["L"].toarray(), levels[-1]["M"].toarray()
    nc = Lc.shape[0]
    Q = np.zeros((nc, nc), order="F")
    mu = np.zeros(nc)
    assert lib.t_pencil(Q.ctypes.data_as(C.POINTER(C.c_double)), mu.ctypes.data_as(C.POINTER(C.c_double))) == 1
    assert np.abs(Q.T @ Mc @ Q - np.eye(nc)).max() < 1e-12
    assert np.abs(Lc @ Q - Mc @ Q @ np.diag(mu)).max() < 1e-10 * np.abs(Lc).max()
    assert mu.min() > -1e-10 * mu.max()  # L_c is positive semidefinite (constants in its null space)
    for sigma in (1e-6, 1e-2, 1.0):
        Ainv = Q @ np.diag(1.0 / (np.maximum(mu, 0.0) + sigma)) @ Q.T
        A = Lc + sigma * Mc
        assert np.abs(Ainv @ A - np.eye(nc)).max() < 1e-8 * max(1.0, 1.0 / (sigma * nc))
