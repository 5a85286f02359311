"""The driver's host-side dense linear algebra (csrc/cr_host_linalg.h), built on
the CPU with g++ and checked against its defining identities and numpy/LAPACK:
the symmetric eigen-decomposition of the residual check and the one-sided
Jacobi SVD of the Galerkin core used by the post-processing."""
import ctypes as C
import os
import shutil
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER_DIR = os.path.join(ROOT, "paper_1808_05510_gb300", "csrc")

WRAPPER = r"""
#include "cr_host_linalg.h"
extern "C" void t_sym_eig(int n, const double* A, double* w, double* V) {
  std::vector<double> a(A, A + (size_t)n * n), ww, vv;
  cr_host::sym_eig(n, a, ww, vv);
  std::copy(ww.begin(), ww.end(), w);
  std::copy(vv.begin(), vv.end(), V);
}
extern "C" void t_svd(int n, const double* A, double* U, double* s, double* V) {
  std::vector<double> a(A, A + (size_t)n * n), ss, vv;
  cr_host::jacobi_svd(n, a, ss, vv);
  std::copy(a.begin(), a.end(), U);
  std::copy(ss.begin(), ss.end(), s);
  std::copy(vv.begin(), vv.end(), V);
}
"""


@pytest.fixture(scope="module")
def lib(tmp_path_factory):
    if shutil.which("g++") is None:
        pytest.skip("g++ not available")
    d = tmp_path_factory.mktemp("hostla")
    src = d / "w.cpp"
    src.write_text(WRAPPER)
    so = d / "libw.so"
    subprocess.run(["g++", "-std=c++17", "-O2", "-shared", "-fPIC", "-I", HEADER_DIR, str(src), "-o", str(so)],
                   check=True)
    L = C.CDLL(str(so))
    dp = np.ctypeslib.ndpointer(dtype=np.float64, flags="F_CONTIGUOUS")
    L.t_sym_eig.argtypes = [C.c_int, dp, dp, dp]
    L.t_svd.argtypes = [C.c_int, dp, dp, dp, dp]
    return L


def sym_eig(lib, A):
    n = A.shape[0]
    w, V = np.zeros(n), np.zeros((n, n), order="F")
    lib.t_sym_eig(n, np.asfortranarray(A), np.asfortranarray(w), V)
    return w, V


def svd(lib, A):
    n = A.shape[0]
    U, s, V = np.zeros((n, n), order="F"), np.zeros(n), np.zeros((n, n), order="F")
    lib.t_svd(n, np.asfortranarray(A), U, np.asfortranarray(s), V)
    return U, s, V


@pytest.mark.parametrize("n,seed", [(1, 0), (5, 1), (28, 2), (60, 3)])
def test_sym_eig(lib, n, seed):
    rng = np.random.default_rng(seed)
    B = rng.standard_normal((n, n))
    A = B @ B.T + np.diag(np.logspace(-8, 0, n))  # symmetric, graded spectrum (a Gram matrix)
    w, V = sym_eig(lib, A)
    nA = np.linalg.norm(A, 2)
    assert np.abs(V.T @ V - np.eye(n)).max() < 1e-13 * n
    assert np.abs(A @ V - V * w).max() < 1e-13 * nA * n
    assert np.abs(np.sort(w) - np.linalg.eigvalsh(A)).max() < 1e-13 * nA * n


@pytest.mark.parametrize("n,seed", [(1, 0), (2, 1), (12, 2), (64, 3), (100, 4)])
def test_jacobi_svd(lib, n, seed):
    rng = np.random.default_rng(seed)
    A = rng.standard_normal((n, n))
    U, s, V = svd(lib, A)
    ref = np.linalg.svd(A, compute_uv=False)
    assert np.all(np.diff(s) <= 0.0) and np.all(s >= 0.0)
    assert np.abs(s - ref).max() < 1e-14 * n * ref[0]
    assert np.abs(U.T @ U - np.eye(n)).max() < 1e-13 * n
    assert np.abs(V.T @ V - np.eye(n)).max() < 1e-13 * n
    assert np.abs(U * s @ V.T - A).max() < 1e-14 * n * ref[0]


def test_jacobi_svd_graded_and_deficient(lib):
    """Graded singular values (1 ... 1e-12) and an exactly rank-deficient core:
    the zero singular value's left vector is completed to an orthonormal set."""
    rng = np.random.default_rng(9)
    n = 20
    Q1 = np.linalg.qr(rng.standard_normal((n, n)))[0]
    Q2 = np.linalg.qr(rng.standard_normal((n, n)))[0]
    sg = np.logspace(0, -12, n)
    A = Q1 @ np.diag(sg) @ Q2.T
    U, s, V = svd(lib, A)
    assert np.abs(s - sg).max() < 1e-14 * n
    assert np.abs(U * s @ V.T - A).max() < 1e-14 * n
    Z = rng.standard_normal((8, 8))
    Z[:, 7] = Z[:, 3]
    Z[:, 6] = 0.0
    U, s, V = svd(lib, Z)
    assert s[-1] == 0.0 or s[-1] < 1e-15 * s[0]
    assert np.abs(U.T @ U - np.eye(8)).max() < 1e-13
    assert np.abs(V.T @ V - np.eye(8)).max() < 1e-13
    assert np.abs(U * s @ V.T - Z).max() < 1e-14 * 8 * s[0]
    # the zero matrix: every left vector comes from the completion
    U, s, V = svd(lib, np.zeros((4, 4)))
    assert not s.any() and np.abs(U.T @ U - np.eye(4)).max() < 1e-15
