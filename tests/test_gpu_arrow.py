"""The device arrowhead eigen-decomposition (csrc/cr_arrow.cu, through
cr_arrow_check) that keeps the eigenbases of U^T L_y U and V^T L_x V up to date
as the Galerkin projection (Eq. Proj_Sylv) grows by one border per greedy step.
Checked against numpy's symmetric eigensolver and the defining identities:
eigenvalues and M W = W diag(mu) to 5e-11 of the matrix's scale (the
eigenvectors are exact for a coupling vector recomputed from the computed
roots, which differs from the given one by rounding), W^T W = I to 1e-13,
including the deflated cases (zero couplings, repeated poles, an empty or a
zero matrix) and the bordering identity it serves."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1808_05510_gb300 import build

    build.build()
    from paper_1808_05510_gb300 import conreg

    conreg.load()
    return conreg


def arrow(lib, d, z, alpha):
    return lib.arrow_check(np.asarray(d, dtype=np.float64), np.asarray(z, dtype=np.float64), float(alpha))


def dense(d, z, alpha):
    n = len(d)
    M = np.zeros((n + 1, n + 1))
    M[:n, :n] = np.diag(d)
    M[:n, n] = z
    M[n, :n] = z
    M[n, n] = alpha
    return M


def check(lib, d, z, alpha, tol=5e-11):
    M = dense(d, z, alpha)
    mu, W = arrow(lib, d, z, alpha)
    scale = max(np.abs(M).max(), 1e-300)
    assert np.all(np.diff(mu) >= -1e-14 * scale)
    assert np.abs(mu - np.linalg.eigvalsh(M)).max() <= tol * scale
    assert np.abs(W.T @ W - np.eye(len(mu))).max() <= 1e-13
    assert np.abs(M @ W - W * mu).max() <= tol * scale


@pytest.mark.parametrize("n", [1, 2, 7, 50, 200])
def test_random_arrowheads(lib, n):
    rng = np.random.default_rng(n)
    d = np.sort(12.0 * rng.random(n) ** 2)
    check(lib, d, 0.3 * rng.standard_normal(n), rng.standard_normal())


def test_deflated_cases(lib):
    rng = np.random.default_rng(5)
    d = np.sort(rng.random(30))
    z = rng.standard_normal(30)
    z[[0, 7, 29]] = 0.0  # uncoupled poles stay eigenpairs
    check(lib, d, z, 0.5)
    d2 = d.copy()
    d2[10] = d2[11] = d2[12] = 0.4  # repeated poles: one coupled combination each
    check(lib, np.sort(d2), z, 0.5)
    check(lib, d, np.zeros(30), -2.0)  # nothing coupled: alpha is an eigenvalue
    mu, W = arrow(lib, np.zeros(0), np.zeros(0), 3.0)  # empty border (eigenvector up to sign)
    assert mu[0] == 3.0 and abs(W[0, 0]) == 1.0
    mu, W = arrow(lib, np.zeros(4), np.zeros(4), 0.0)  # zero matrix
    assert np.all(mu == 0.0) and np.array_equal(W, np.eye(5))


def test_bordering_keeps_the_eigenbasis(lib):
    """Grow a symmetric matrix one border at a time from its 1 x 1 corner, as
    U^T L U grows with U: the basis follows and diagonalises every leading
    block, like a fresh eigen-decomposition."""
    rng = np.random.default_rng(9)
    B = rng.standard_normal((40, 40))
    A = B @ B.T / 40 + np.diag(np.linspace(0, 3, 40))
    Q = np.ones((1, 1))
    lam = np.array([A[0, 0]])
    for j in range(1, 40):
        z = Q.T @ A[:j, j]
        mu, W = arrow(lib, lam, z, A[j, j])
        Qe = np.zeros((j + 1, j + 1))
        Qe[:j, :j] = Q
        Qe[j, j] = 1.0
        Q, lam = Qe @ W, mu
    assert np.abs(Q.T @ A @ Q - np.diag(lam)).max() <= 1e-11 * np.abs(A).max()
    assert np.abs(lam - np.linalg.eigvalsh(A)).max() <= 1e-11 * np.abs(A).max()


def test_bases_follow_a_growing_projection(lib):
    """Three hundred borders of U^T L U for a 2-D Laplacian and an orthonormal U
    that grows by one smooth column at a time, the way the greedy rank grows:
    the basis updated border by border stays orthonormal and diagonalizes the
    projected matrix, with eigenvalues equal to numpy's.  Each border adds
    rounding of order the deflation threshold (8 eps of the scale), so the
    error grows about linearly with the borders: the bound is 64 eps of the
    scale per border."""
    import scipy.sparse as sp

    nside = 40
    T = sp.diags([-np.ones(nside - 1), 2 * np.ones(nside), -np.ones(nside - 1)], [-1, 0, 1])
    L = (sp.kron(T, sp.identity(nside)) + sp.kron(sp.identity(nside), T)).tocsr()
    n = L.shape[0]
    rng = np.random.default_rng(3)
    steps = 300
    U = np.zeros((n, steps))
    Q = np.zeros((0, 0))
    lam = np.zeros(0)
    A = np.zeros((0, 0))
    for q in range(steps):
        w = rng.standard_normal(n)
        for _ in range(2):  # smooth it a little, like an ALS factor
            w = w - 0.2 * (L @ w)
        w -= U[:, :q] @ (U[:, :q].T @ w)
        w -= U[:, :q] @ (U[:, :q].T @ w)
        U[:, q] = w / np.linalg.norm(w)
        a = U[:, :q + 1].T @ (L @ U[:, q])
        A = np.block([[A, a[:q, None]], [a[None, :q], a[q:q + 1, None]]])
        mu, W = arrow(lib, lam, Q.T @ a[:q], a[q])
        Qb = np.zeros((q + 1, q + 1))
        Qb[:q, :q] = Q
        Qb[q, q] = 1.0
        Q = Qb @ W
        lam = mu
    scale = np.abs(A).max()
    bound = steps * 64 * np.finfo(float).eps
    assert np.abs(Q.T @ Q - np.eye(steps)).max() < bound
    assert np.abs(Q.T @ A @ Q - np.diag(lam)).max() < bound * scale
    assert np.abs(lam - np.linalg.eigvalsh(A)).max() < bound * scale
