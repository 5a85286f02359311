"""Pins for the post-processing oracle (SVD of the solution, error measures,
nonnegative projection).  Each test ties ``oracle.post`` to something other than
itself: the SVD of the dense W, the defining properties of a Euclidean
projection onto a convex cone, closed-form distances, a brute-force loop over a
tiny matrix, and the toy-brain statements of Sec. 4."""
import json
import math
import os

import numpy as np
import pytest

from oracle import Oracle
from oracle import post
from paper_1808_05510_gb300 import synth

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def orthonormal(rng, n, j):
    q, _ = np.linalg.qr(rng.standard_normal((n, j)))
    return q


def factors(seed=0, ny=37, nx=29, j=6):
    rng = np.random.default_rng(seed)
    return orthonormal(rng, ny, j), rng.standard_normal((j, j)), orthonormal(rng, nx, j)


# --------------------------------------------------------------------------- SVD (Sec. 4)
@pytest.mark.parametrize("seed,ny,nx,j", [(0, 37, 29, 6), (1, 50, 50, 12), (2, 9, 40, 1)])
def test_svd_matches_dense_svd(seed, ny, nx, j):
    U, Z, V = factors(seed, ny, nx, j)
    W = U @ Z @ V.T
    Uh, s, Vh = post.solution_svd(U, Z, V)
    sd = np.linalg.svd(W, compute_uv=False)  # the dense route, independent of the factors
    assert np.all(np.diff(s) <= 0.0)
    assert np.abs(s - sd[:j]).max() <= 1e-12 * sd[0]
    assert np.abs(sd[j:]).max(initial=0.0) <= 1e-12 * sd[0]  # rank j
    assert np.abs(Uh.T @ Uh - np.eye(j)).max() < 1e-12
    assert np.abs(Vh.T @ Vh - np.eye(j)).max() < 1e-12
    assert np.abs(Uh @ np.diag(s) @ Vh.T - W).max() <= 1e-12 * np.abs(W).max()
    # each singular pair is one of W's: W v^_k = s_k u^_k and W^T u^_k = s_k v^_k
    assert np.abs(W @ Vh - Uh * s).max() <= 1e-12 * sd[0]
    assert np.abs(W.T @ Uh - Vh * s).max() <= 1e-12 * sd[0]


def test_svd_of_diagonal_core_is_a_permutation():
    """With Z diagonal the SVD only sorts and signs the given columns."""
    rng = np.random.default_rng(3)
    U, V = orthonormal(rng, 20, 4), orthonormal(rng, 15, 4)
    d = np.array([0.5, -3.0, 2.0, 1e-3])
    Uh, s, Vh = post.solution_svd(U, np.diag(d), V)
    assert np.allclose(s, [3.0, 2.0, 0.5, 1e-3], rtol=0, atol=1e-15)
    order = [1, 2, 0, 3]
    for k, c in enumerate(order):
        assert abs(abs(Uh[:, k] @ U[:, c]) - 1.0) < 1e-13
        assert abs(abs(Vh[:, k] @ V[:, c]) - 1.0) < 1e-13


# --------------------------------------------------------------------------- projection (Sec. 4)
def test_projection_is_the_nearest_nonnegative_matrix():
    """max(0, W) is the Euclidean projection onto the nonnegative cone: it is
    nonnegative, idempotent, complementary (<W - P, P> = 0, W - P <= 0) and no
    sampled nonnegative matrix is closer."""
    rng = np.random.default_rng(4)
    W = rng.standard_normal((12, 9))
    P = post.project_nonneg(W)
    assert (P >= 0.0).all()
    assert np.array_equal(post.project_nonneg(P), P)
    assert abs(np.sum((W - P) * P)) == 0.0
    assert ((W - P) <= 0.0).all()
    best = np.linalg.norm(W - P)
    for _ in range(200):
        M = np.abs(P + 0.3 * rng.standard_normal(W.shape))
        assert np.linalg.norm(W - M) >= best
    # projection is non-expansive towards any nonnegative target
    T = np.abs(rng.standard_normal(W.shape))
    assert np.linalg.norm(P - T) <= np.linalg.norm(W - T)


def test_report_counts_by_brute_force():
    rng = np.random.default_rng(5)
    U, Z, V = factors(5, 8, 7, 3)
    r = post.solution_report(U, Z, V)
    W = U @ Z @ V.T
    n_neg, wmin, wmax, neg2, w2 = 0, math.inf, -math.inf, 0.0, 0.0
    for i in range(W.shape[0]):
        for k in range(W.shape[1]):
            x = float(W[i, k])
            wmin, wmax = min(wmin, x), max(wmax, x)
            w2 += x * x
            if x < 0.0:
                n_neg += 1
                neg2 += x * x
    assert r["n_negative"] == n_neg and r["entries"] == 56
    assert r["w_min"] == wmin and r["w_max"] == wmax
    assert math.isclose(r["w_fro2"], w2, rel_tol=1e-13) and math.isclose(r["neg_fro2"], neg2, rel_tol=1e-13)
    # W* = 0: the distance is |W| itself, and E_rel is undefined
    assert math.isclose(r["diff_fro2"], w2, rel_tol=1e-13) and r["ref_fro2"] == 0.0 and math.isnan(r["rel"])
    assert rng is not None


# --------------------------------------------------------------------------- error measures (Sec. 3)
def test_error_measures_closed_forms():
    U, Z, V = factors(6, 30, 20, 5)
    W = U @ Z @ V.T
    same = post.solution_report(U, Z, V, ref=(U, Z, V))
    assert same["diff_fro2"] == 0.0 and same["rms"] == 0.0 and same["rel"] == 0.0
    # W* = -W: |W - W*| = 2|W|, E_rel = 2; orthonormal U*, V*: |W*|_F = |Z*|_F
    neg = post.solution_report(U, Z, V, ref=(U, -Z, V))
    assert math.isclose(neg["rel"], 2.0, rel_tol=1e-13)
    assert math.isclose(neg["ref_fro2"], float(np.sum(Z * Z)), rel_tol=1e-12)
    assert math.isclose(neg["rms"], 2.0 * np.linalg.norm(W) / math.sqrt(600), rel_tol=1e-13)
    # W* = W + c e_i e_k^T (a rank-one border of the factors): distance |c| in every norm
    i, k, c = 7, 3, -0.25
    ei, ek = np.eye(30)[:, [i]], np.eye(20)[:, [k]]
    Zr = np.zeros((6, 6))
    Zr[:5, :5], Zr[5, 5] = Z, c
    r = post.solution_report(U, Z, V, ref=(np.hstack([U, ei]), Zr, np.hstack([V, ek])))
    assert math.isclose(r["diff_fro2"], c * c, rel_tol=1e-10)
    assert math.isclose(r["diff_maxabs"], abs(c), rel_tol=1e-10)
    assert math.isclose(r["rms"], abs(c) / math.sqrt(600), rel_tol=1e-10)


def test_projected_report_compares_the_projection():
    U, Z, V = factors(7, 25, 25, 4)
    W = U @ Z @ V.T
    r = post.solution_report(U, Z, V, nonneg=True, ref=(U, Z, V))
    # |max(0, W) - W| = |min(0, W)|: the distance equals the negative mass
    assert math.isclose(r["diff_fro2"], r["neg_fro2"], rel_tol=1e-12)
    assert math.isclose(r["diff_maxabs"], -min(W.min(), 0.0), rel_tol=1e-12)
    assert (r["W_out"] >= 0.0).all()


def test_rank_zero_solution():
    U, V = np.zeros((6, 0)), np.zeros((4, 0))
    r = post.solution_report(U, np.zeros((0, 0)), V)
    assert r["n_negative"] == 0 and r["w_min"] == 0.0 and r["w_max"] == 0.0 and r["diff_fro2"] == 0.0
    Uh, s, Vh = post.solution_svd(U, np.zeros((0, 0)), V)
    assert s.size == 0 and Uh.shape == (6, 0) and Vh.shape == (4, 0)


# --------------------------------------------------------------------------- toy brain (Secs. 3.1, 4)
def test_paper_toy_nearly_nonnegative():
    """Sec. 4: the toy's rank-40 solution is nearly nonnegative; its few negative
    entries sit in the lower-left corner of W, where the truth is about zero, and
    projecting them away moves W towards the (nonnegative) truth."""
    gold = json.load(open(os.path.join(GOLD, "paper_toy_nonneg.json")))
    p = synth.paper_toy()
    o = Oracle.from_problem(p)
    res = o.greedy(r_max=40, tau=1e-7)
    assert res.U.shape[1] == 40
    r = post.solution_report(res.U, res.Z, res.V, nonneg=True, ref=None)
    W = post.dense_w(res.U, res.Z, res.V)
    Wt = p.W_true
    assert (Wt >= 0.0).all()
    assert 0 < r["n_negative"] <= gold["band_negative_fraction_max"] * r["entries"]
    neg = W < 0.0
    assert Wt[neg].max() <= gold["band_truth_at_negatives_max_rel"] * Wt.max()
    ii, kk = np.nonzero(neg)
    ny, nx = W.shape
    assert np.mean((ii >= ny // 2) & (kk < nx // 2)) >= gold["band_lower_left_fraction_min"]
    assert post.rms_error(r["W_out"], Wt) <= post.rms_error(W, Wt)
    assert math.isclose(r["neg_fro2"], float(np.sum(np.minimum(W, 0.0) ** 2)), rel_tol=1e-12)
