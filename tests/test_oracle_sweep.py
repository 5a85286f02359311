"""Pins for the held-out scoring of the lambda x fold sweep and for its input
structure: a hand-computed example, the value at W = 0, zero error on
noiseless data of a known W, agreement with the data term of the objective
(Eq. obj_fun), and the fold partition's invariants."""
import numpy as np

from oracle import Oracle
from paper_1808_05510_gb300 import synth


def test_cv_error_hand_example():
    # W = U Z V^T = [[2, 2], [0, 0], [0, 0]], x = (1, 1): W x = (4, 0, 0);
    # y = (1, 2, 3) with the third entry unobserved: residual (3, -2, 0)
    U = np.array([[1.0], [0.0], [0.0]])
    Z = np.array([[2.0]])
    V = np.array([[1.0], [1.0]])
    num, den = Oracle.cv_error(U, Z, V, np.array([[1.0], [1.0]]), np.array([[1.0], [2.0], [3.0]]),
                               np.array([[1], [1], [0]], dtype=np.uint8))
    assert num == 13.0 and den == 5.0


def test_cv_error_at_zero_and_on_noiseless_data():
    p = synth.toy2d(seed=3)
    rng = np.random.default_rng(0)
    Xt = p.X[:, :3]
    Om = (rng.random((p.ny, 3)) > 0.2).astype(np.uint8)
    Yt = (p.W_true @ Xt) * Om
    num0, den0 = Oracle.cv_error(np.zeros((p.ny, 1)), np.zeros((1, 1)), np.zeros((p.nx, 1)), Xt, Yt, Om)
    assert num0 == den0 > 0
    U, s, Vt = np.linalg.svd(p.W_true)
    num, den = Oracle.cv_error(U, np.diag(s), Vt.T, Xt, Yt, Om)
    assert num <= 1e-24 * den


def test_cv_error_is_data_term_of_objective():
    """On the fitted columns, num = 2 J(W) - lambda |L_y W + W L_x^T|^2."""
    p = synth.rect2d()
    o = Oracle.from_problem(p)
    rng = np.random.default_rng(4)
    U, Z, V = rng.standard_normal((p.ny, 3)), rng.standard_normal((3, 3)), rng.standard_normal((p.nx, 3))
    W = U @ Z @ V.T
    S = o.Ly @ W + (o.Lx @ W.T).T
    num, _ = Oracle.cv_error(U, Z, V, p.X, p.Y, p.Omega)
    assert abs(num - (2.0 * o.J(W) - p.lam * np.sum(S * S))) <= 1e-12 * num


def test_fold_partition_and_members():
    for (m, k, lo, hi) in ((126, 5, 20, 30), (10, 2, 4, 6), (7, 7, 1, 1)):
        folds = synth.fold_partition(m, k, lo, hi, seed=3)
        assert len(folds) == k
        allc = np.concatenate(folds)
        assert sorted(allc.tolist()) == list(range(m))
        assert all(lo <= len(f) <= hi for f in folds)
        again = synth.fold_partition(m, k, lo, hi, seed=3)
        assert all(np.array_equal(a, b) for a, b in zip(folds, again))
    folds = synth.fold_partition(126)
    assert len({len(f) for f in folds}) > 1  # uneven injection counts
    lams = synth.lambda_grid()
    assert len(lams) == 16 and lams[0] == 1.0 and abs(lams[-1] - 1e6) <= 1e-6
    assert np.allclose(np.diff(np.log10(lams)), 0.4)
    mem = synth.sweep_members(126, lams, folds)
    assert len(mem) == 80
    for lam, fit, test in mem:
        assert len(np.intersect1d(fit, test)) == 0 and len(fit) + len(test) == 126
