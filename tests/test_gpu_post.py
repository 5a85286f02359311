"""GPU parity of the post-processing calls (cr_svd_factors, cr_solution_report)
against the CPU float64 oracle, on seeded factors loaded with cr_set_factors,
plus properties of the GPU's own solutions that hold at any size.

Tolerances.  Both sides are float64.  Entries of W = U Z V^T and of the
singular factors differ by summation order only: 1e-12 relative to the largest
entry (j <= 64 terms).  Sums of squares over ny * nx entries: 1e-12 relative.
Singular values: the one-sided Jacobi method is accurate to a few eps relative
to sigma_max, so 1e-13 * sigma_max.  Whether an entry is negative is decided
in float64 on both sides; entries within 1e-13 * max|W| of zero may fall
either way, so the count is checked against the oracle's counts on both sides
of that band.
"""
import math

import numpy as np
import pytest

from oracle import post
from paper_1808_05510_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def cr():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1808_05510_gb300 import build

    build.build()
    from paper_1808_05510_gb300 import conreg

    conreg.load()
    return conreg


def seeded_factors(ny, nx, j, seed):
    """Orthonormal U (ny x j), V (nx x j) and a Gaussian core Z (j x j)."""
    rng = np.random.default_rng(seed)
    U = np.linalg.qr(rng.standard_normal((ny, j)))[0]
    V = np.linalg.qr(rng.standard_normal((nx, j)))[0]
    return U, rng.standard_normal((j, j)), V


PROBS = {
    "paper_toy": synth.paper_toy,       # 200 x 200: three full tiles and a ragged tail
    "rect2d": synth.rect2d,             # ny != nx, both under one tile
    "masked3d": synth.masked3d,
}


@pytest.mark.parametrize("name,j", [("paper_toy", 12), ("rect2d", 7), ("masked3d", 20), ("paper_toy", 1)])
def test_svd_factors_match_oracle(cr, name, j):
    p = PROBS[name]()
    U, Z, V = seeded_factors(p.ny, p.nx, j, 100 + j)
    Uo, so, Vo = post.solution_svd(U, Z, V)
    with cr.ConReg.from_problem(p, r_cap=max(j, 2)) as g:
        g.cr_set_factors(U, Z, V)
        Uh, s, Vh = g.cr_svd_factors()
    assert np.abs(s - so).max() <= 1e-13 * so[0]
    # singular pairs: unique up to one common sign per pair (the values are simple here)
    assert j == 1 or np.abs(np.diff(so)).min() > 1e-3 * so[0]  # simple, well separated
    for k in range(j):
        sg = np.sign(Uh[:, k] @ Uo[:, k])
        assert np.abs(sg * Uh[:, k] - Uo[:, k]).max() <= 1e-10
        assert np.abs(sg * Vh[:, k] - Vo[:, k]).max() <= 1e-10
    W = U @ Z @ V.T
    assert np.abs(Uh @ np.diag(s) @ Vh.T - W).max() <= 1e-12 * np.abs(W).max()
    assert np.abs(Uh.T @ Uh - np.eye(j)).max() <= 1e-12
    assert np.abs(Vh.T @ Vh - np.eye(j)).max() <= 1e-12


def test_svd_factors_rank_deficient_core(cr):
    """A core with two equal columns has a zero singular value: the left vector
    for it is completed, so U^ stays orthonormal and W is still reproduced."""
    p = synth.masked3d()
    j = 6
    rng = np.random.default_rng(7)
    U = np.linalg.qr(rng.standard_normal((p.ny, j)))[0]
    V = np.linalg.qr(rng.standard_normal((p.nx, j)))[0]
    Z = rng.standard_normal((j, j))
    Z[:, 5] = Z[:, 2]
    so = post.solution_svd(U, Z, V)[1]
    with cr.ConReg.from_problem(p, r_cap=j) as g:
        g.cr_set_factors(U, Z, V)
        Uh, s, Vh = g.cr_svd_factors()
    assert np.abs(s - so).max() <= 1e-13 * so[0]
    assert s[-1] <= 1e-14 * s[0]
    assert np.abs(Uh.T @ Uh - np.eye(j)).max() <= 1e-12
    assert np.abs(Vh.T @ Vh - np.eye(j)).max() <= 1e-12
    W = U @ Z @ V.T
    assert np.abs(Uh @ np.diag(s) @ Vh.T - W).max() <= 1e-12 * np.abs(W).max()


def check_report(r, o, W_max):
    assert r["entries"] == o["entries"]
    for k in ("w_fro2", "neg_fro2", "ref_fro2", "diff_fro2"):
        assert abs(r[k] - o[k]) <= 1e-12 * max(abs(o[k]), 1e-300), k
    for k in ("w_min", "w_max", "diff_maxabs"):
        assert abs(r[k] - o[k]) <= 1e-12 * W_max, k
    assert abs(r["rms"] - o["rms"]) <= 1e-12 * max(o["rms"], 1e-300)
    if math.isnan(o["rel"]):
        assert math.isnan(r["rel"])
    else:
        assert abs(r["rel"] - o["rel"]) <= 1e-12 * o["rel"]


@pytest.mark.parametrize("nonneg", [False, True])
@pytest.mark.parametrize("name,j,jr", [("paper_toy", 12, 0), ("paper_toy", 9, 15), ("rect2d", 5, 3),
                                        ("masked3d", 20, 8)])
def test_solution_report_matches_oracle(cr, name, j, jr, nonneg):
    p = PROBS[name]()
    U, Z, V = seeded_factors(p.ny, p.nx, j, 200 + j)
    ref = None
    if jr:
        rng = np.random.default_rng(300 + jr)
        # a reference with general (not orthonormal) factors
        ref = (rng.standard_normal((p.ny, jr)), rng.standard_normal((jr, jr)) / jr,
               rng.standard_normal((p.nx, jr)))
    o = post.solution_report(U, Z, V, nonneg=nonneg, ref=ref)
    with cr.ConReg.from_problem(p, r_cap=j) as g:
        g.cr_set_factors(U, Z, V)
        r = g.cr_solution_report(nonneg=nonneg, ref=ref, want_w=True)
        r2 = g.cr_solution_report(nonneg=nonneg, ref=ref, want_w=False)
    W = post.dense_w(U, Z, V)
    wmax = np.abs(W).max()
    check_report(r, o, wmax)
    band = 1e-13 * wmax
    assert int((W < -band).sum()) <= r["n_negative"] <= int((W < band).sum())
    assert np.abs(r["W_out"] - o["W_out"]).max() <= 1e-12 * wmax
    if nonneg:
        assert (r["W_out"] >= 0.0).all()
    # the pass without the host copy is the same pass: identical statistics
    for k in ("n_negative", "w_min", "w_max", "w_fro2", "neg_fro2", "ref_fro2", "diff_fro2", "diff_maxabs"):
        assert r2[k] == r[k], k


def test_solution_report_rank_zero(cr):
    p = synth.rect2d()
    with cr.ConReg.from_problem(p, r_cap=4) as g:
        r = g.cr_solution_report(nonneg=True, want_w=True)
    assert r["entries"] == p.ny * p.nx and r["n_negative"] == 0
    assert r["w_min"] == 0.0 and r["w_max"] == 0.0 and r["diff_fro2"] == 0.0 and math.isnan(r["rel"])
    assert not r["W_out"].any()


def test_solution_report_rejects_bad_arguments(cr):
    """Through the ABI directly (the binding always passes valid sizes)."""
    import ctypes as C

    p = synth.rect2d()
    st = cr.cr_solution_stats()
    buf = np.zeros(p.ny * p.nx + 16)
    ptr = buf.ctypes.data_as(C.POINTER(C.c_double))
    with cr.ConReg.from_problem(p, r_cap=4) as g:
        call = g._lib.cr_solution_report
        assert call(g.h, 0, -1, None, 1, None, 1, None, 1, None, 1, C.byref(st)) == cr.CR_EINVAL
        assert call(g.h, 0, 2, None, p.ny, None, 2, None, p.nx, None, 1, C.byref(st)) == cr.CR_EINVAL
        assert call(g.h, 0, 2, ptr, p.ny - 1, ptr, 2, ptr, p.nx, None, 1, C.byref(st)) == cr.CR_EINVAL
        assert call(g.h, 0, 0, None, 1, None, 1, None, 1, ptr, p.ny - 1, C.byref(st)) == cr.CR_EINVAL
        assert call(g.h, 0, 0, None, 1, None, 1, None, 1, None, 1, None) == cr.CR_EINVAL
        assert call(g.h, 0, 0, None, 1, None, 1, None, 1, ptr, p.ny, C.byref(st)) == cr.CR_OK


def test_visual_cortex_full_size_blocks_and_determinism(cr):
    """Bench-sized W (7,530 x 7,530, 453 MB): the host copy goes through two
    column blocks of the 256 MiB device buffer.  Every entry is compared with the
    oracle's dense W; repeated passes agree bit for bit."""
    p = synth.visual_cortex()
    j, jr = 64, 24
    U, Z, V = seeded_factors(p.ny, p.nx, j, 401)
    rng = np.random.default_rng(402)
    ref = (np.linalg.qr(rng.standard_normal((p.ny, jr)))[0], rng.standard_normal((jr, jr)),
           np.linalg.qr(rng.standard_normal((p.nx, jr)))[0])
    o = post.solution_report(U, Z, V, nonneg=True, ref=ref)
    with cr.ConReg.from_problem(p, r_cap=j) as g:
        g.cr_set_factors(U, Z, V)
        r = g.cr_solution_report(nonneg=True, ref=ref, want_w=True)
        again = g.cr_solution_report(nonneg=True, ref=ref, want_w=True)
        one = g.cr_solution_report(nonneg=True, ref=ref, want_w=False)  # one launch over all columns
        Uh, s, Vh = g.cr_svd_factors()
    W_max = max(abs(o["w_min"]), abs(o["w_max"]))
    check_report(r, o, W_max)
    check_report(one, o, W_max)
    assert np.abs(r["W_out"] - o["W_out"]).max() <= 1e-12 * W_max
    assert np.array_equal(again["W_out"], r["W_out"])
    for k in ("n_negative", "w_min", "w_max", "w_fro2", "neg_fro2", "ref_fro2", "diff_fro2", "diff_maxabs"):
        assert again[k] == r[k], k
    # the blocked and the one-launch pass split the tiles differently: same
    # entries, extremes and count; sums equal up to their order
    for k in ("n_negative", "w_min", "w_max", "diff_maxabs"):
        assert one[k] == r[k], k
    so = post.solution_svd(U, Z, V)[1]
    assert np.abs(s - so).max() <= 1e-13 * so[0]


def test_solved_problem_properties(cr):
    """Properties of the GPU's own solution that hold at any size: |W|_F = |Z|_F
    and sum sigma^2 = |Z|_F^2 (orthonormal bases); compared with itself under
    the projection, the distance is exactly the negative mass."""
    p = synth.visual_cortex()
    with cr.ConReg.from_problem(p, r_cap=24) as g:
        g.cr_solve(16, 1e-9, 0.0)
        j = g.cr_get_rank()
        U, Z, V = g.cr_get_factors()
        r = g.cr_solution_report(nonneg=True, ref=(U, Z, V))
        plain = g.cr_solution_report()
        Uh, s, Vh = g.cr_svd_factors()
    z2 = float(np.sum(Z * Z))
    assert abs(plain["w_fro2"] - z2) <= 1e-10 * z2
    assert abs(float(np.sum(s * s)) - z2) <= 1e-12 * z2
    assert abs(r["diff_fro2"] - r["neg_fro2"]) <= 1e-12 * max(r["neg_fro2"], 1e-300) + 1e-30
    assert abs(r["diff_maxabs"] - max(-r["w_min"], 0.0)) <= 1e-12 * max(abs(r["w_min"]), 1e-300)
    assert abs(r["rms"] - math.sqrt(r["diff_fro2"] / (p.ny * p.nx))) <= 1e-14 * max(r["rms"], 1e-300)
    assert r["n_negative"] == plain["n_negative"]
    assert j >= 8 and np.abs(Uh.T @ Uh - np.eye(j)).max() <= 1e-10


def test_paper_toy_nearly_nonnegative_on_gpu(cr):
    """Sec. 4's statements about the toy's rank-40 solution, on the GPU path: few
    negative entries, all in the lower-left corner, and the projection moves W
    towards the nonnegative truth."""
    p = synth.paper_toy()
    Wt = p.W_true
    with cr.ConReg.from_problem(p, r_cap=40) as g:
        g.cr_solve(40, 1e-7, 0.0)
        assert g.cr_get_rank() == 40
        r = g.cr_solution_report(nonneg=False, want_w=True)
        U, Z, V = g.cr_get_factors()
        # W_true as a reference: its exact SVD factors (dense, n = 200)
        Ut, st, Vtt = np.linalg.svd(Wt)
        proj = g.cr_solution_report(nonneg=True, ref=(Ut, np.diag(st), Vtt.T))
        plain = g.cr_solution_report(nonneg=False, ref=(Ut, np.diag(st), Vtt.T))
    W = r["W_out"]
    assert 0 < r["n_negative"] <= 0.05 * r["entries"]
    ii, kk = np.nonzero(W < 0.0)
    assert np.mean((ii >= p.ny // 2) & (kk < p.nx // 2)) >= 0.9
    assert proj["rms"] <= plain["rms"]
    assert 0.04 <= plain["rms"] <= 0.12  # Table tab:test band of E(W_40, W_true)
