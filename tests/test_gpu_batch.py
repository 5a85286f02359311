"""The lambda x fold sweep (cr_solve_batch) against the float64 oracle.

Every member is an independent greedy solve of a sub-problem (the member's
injection columns, its lambda), so each member's W must match the oracle's
greedy run on that sub-problem exactly as a single solve does (1e-9 relative,
deterministic mode: two ALS sweeps, PCG to 1e-13), and its held-out error must
match the oracle's cv_error on the oracle's factors.  Running members
concurrently must not change any result."""
import numpy as np
import pytest

from oracle import Oracle
from paper_1808_05510_gb300 import synth

pytestmark = pytest.mark.gpu

R = 4
DET = dict(pcg_tol=1e-13, pcg_maxit=50000, als_sweeps=2)


@pytest.fixture(scope="module")
def cr():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1808_05510_gb300 import build

    build.build()
    from paper_1808_05510_gb300 import conreg

    conreg.load()
    return conreg


@pytest.fixture(scope="module")
def data():
    p = synth.masked3d(seed=31, box=10, n_target=300, m=10)
    folds = synth.fold_partition(10, 2, 4, 6, seed=2)
    members = synth.sweep_members(10, [5.0, 200.0, 1e5], folds)
    return p, members


def rel(a, b):
    return np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(b), 1e-300)


def test_batch_members_match_oracle(cr, data):
    p, members = data
    res, kept = cr.solve_batch(p, members, r_max=R, tau=1e-13, concurrency=4, keep=True, **DET)
    try:
        assert len({r["slot"] for r in res}) > 1  # members really ran on several workers
        for (lam, fit, test), r, g in zip(members, res, kept):
            assert r["status"] == 0 and r["rank"] == R
            o = Oracle.from_problem(synth.member_problem(p, lam, fit))
            ref = o.greedy(r_max=R, tau=1e-13, als_sweeps=2, galerkin_tol=1e-14)
            U, Z, V = g.cr_get_factors()
            assert rel(U @ Z @ V.T, ref.U @ ref.Z @ ref.V.T) < 1e-9
            num, den = Oracle.cv_error(ref.U, ref.Z, ref.V, p.X[:, test], p.Y[:, test], p.Omega[:, test])
            assert abs(r["cv_num"] - num) <= 1e-8 * num
            assert abs(r["cv_den"] - den) <= 1e-12 * den
            assert abs(r["relres"] - ref.steps[-1].relres) <= 1e-8 * ref.steps[-1].relres
    finally:
        for g in kept:
            g.close()


def test_batch_concurrency_does_not_change_results(cr, data):
    p, members = data
    runs = [cr.solve_batch(p, members, r_max=R, tau=1e-13, concurrency=c, galerkin_ctas=8, **DET) for c in (1, 4)]
    for a, b in zip(*runs):
        for key in ("rank", "relres", "J", "cv_num", "cv_den", "pcg_iters", "cg_iters"):
            assert a[key] == b[key], key


def test_batch_mixed_form_close_to_fp64(cr, data):
    """The sweep in the mixed form (float32 sub-solves and inner Galerkin CG,
    float64 refinement): relative residual and held-out error within 1e-4 of
    the float64 sweep (sub-solves and Galerkin solves are refined to the float64
    tolerances; what remains is float32 rounding in the inner solves)."""
    p, members = data
    f64 = cr.solve_batch(p, members, r_max=R, tau=1e-12, concurrency=4)
    mix = cr.solve_batch(p, members, r_max=R, tau=1e-12, concurrency=4, precision=cr.CR_MIXED)
    for a, b in zip(f64, mix):
        assert b["status"] == 0 and b["rank"] == a["rank"]
        assert abs(b["relres"] - a["relres"]) <= 1e-4 * a["relres"]
        assert abs(b["cv_num"] - a["cv_num"]) <= 1e-4 * a["cv_num"]


def test_batch_edge_cases(cr, data):
    p, members = data
    assert cr.solve_batch(p, [], r_max=R) == []
    lam, fit, _ = members[0]
    res = cr.solve_batch(p, [(lam, fit, None)], r_max=2, concurrency=3)
    assert res[0]["status"] == 0 and res[0]["cv_num"] == 0.0 and res[0]["cv_den"] == 0.0
    with pytest.raises(cr.ConRegError):
        cr.solve_batch(p, [(lam, np.array([0, 99]), None)], r_max=2)
    with pytest.raises(cr.ConRegError):
        cr.solve_batch(p, [(-1.0, fit, None)], r_max=2)


def test_autotune_and_cv_summary(cr, data):
    from paper_1808_05510_gb300 import sweep

    p, members = data
    cands = ((1, 16), (3, 8))
    shape = sweep.autotune(p, members, r_probe=1, candidates=cands)
    assert (shape["concurrency"], shape["cluster_size"]) in cands and len(shape["table"]) == 2
    out = sweep.run(p, members, r_max=2, tune=False)
    curve = out["cv_by_lambda"]
    assert set(curve) == {m[0] for m in members}
    lam = members[0][0]
    rs = [r for m, r in zip(members, out["results"]) if m[0] == lam]
    assert abs(curve[lam] - sum(r["cv_num"] for r in rs) / sum(r["cv_den"] for r in rs)) <= 1e-15 * curve[lam]
    assert out["best_lambda"] == min(curve, key=curve.get)
