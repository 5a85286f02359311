"""GPU checks of the mixed-precision form (float32 sub-solves with float64 inner
products; float32 inner Galerkin CG under float64 iterative refinement).

Stated per-result error against float64:
* ALS sub-solves: float64 iterative refinement around the float32 PCG reaches
  the float64 form's tolerance, so the relative residual measured in float64
  by the oracle is <= 2 pcg_tol (pcg_tol = 1e-10), also at lambda = 1e7 where
  float32 alone cannot resolve the system.
* Galerkin projection: refined to the requested float64 tolerance, so Z agrees
  with the oracle's float64 Galerkin solution to 1e-9 relative.
* Greedy runs: J(W_j) non-increasing and U^T R_j V = 0 (Galerkin condition) to
  1e-9 of |D|, with R_j formed densely by the oracle.
"""
import numpy as np
import pytest

from oracle import Oracle
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


@pytest.fixture(scope="module", params=["toy2d", "masked3d"])
def prob(request):
    p = synth.toy2d() if request.param == "toy2d" else synth.masked3d()
    return p, Oracle.from_problem(p)


def rel(a, b):
    return np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(b), 1e-300)


def test_mixed_subsolve_residuals(cr, prob):
    p, o = prob
    rng = np.random.default_rng(31)
    v = synth.random_unit(p.nx, 32)
    u = synth.random_unit(p.ny, 33)
    rhs_u = rng.standard_normal(p.ny)
    rhs_v = rng.standard_normal(p.nx)
    with cr.ConReg.from_problem(p, r_cap=4, precision=cr.CR_MIXED) as g:
        uh, _ = g.cr_solve_u(v, rhs_u)
        vh, _ = g.cr_solve_v(u, rhs_v)
    Ah = o.A_hat(v)
    assert np.linalg.norm(Ah @ uh - rhs_u) <= 2e-10 * np.linalg.norm(rhs_u)
    S, s = o.B_hat(u)
    Bv = S @ vh + p.X @ (s * (p.X.T @ vh))
    assert np.linalg.norm(Bv - rhs_v) <= 2e-10 * np.linalg.norm(rhs_v)


@pytest.mark.parametrize("lam", [1e4, 1e7])
def test_mixed_subsolves_at_large_lambda(cr, lam):
    """Very ill-conditioned sub-systems: refinement (with the float64 hand-over
    when float32 stalls) still meets the float64 tolerance."""
    import dataclasses

    p = dataclasses.replace(synth.masked3d(), lam=lam)
    o = Oracle.from_problem(p)
    rng = np.random.default_rng(35)
    v = synth.random_unit(p.nx, 36)
    u = synth.random_unit(p.ny, 37)
    rhs_u = rng.standard_normal(p.ny)
    rhs_v = rng.standard_normal(p.nx)
    with cr.ConReg.from_problem(p, r_cap=4, precision=cr.CR_MIXED, pcg_maxit=200000) as g:
        uh, _ = g.cr_solve_u(v, rhs_u)
        vh, _ = g.cr_solve_v(u, rhs_v)
        st = g.cr_get_stats()
    print("handovers", st["mixed_handovers"])
    assert np.linalg.norm(o.A_hat(v) @ uh - rhs_u) <= 2e-10 * np.linalg.norm(rhs_u)
    S, s = o.B_hat(u)
    assert np.linalg.norm(S @ vh + p.X @ (s * (p.X.T @ vh)) - rhs_v) <= 2e-10 * np.linalg.norm(rhs_v)


def test_mixed_galerkin_refined_to_fp64(cr, prob):
    p, o = prob
    j = 6
    rng = np.random.default_rng(34)
    U, _ = np.linalg.qr(rng.standard_normal((o.ny, j)))
    V, _ = np.linalg.qr(rng.standard_normal((o.nx, j)))
    Z0 = 1e-3 * rng.standard_normal((j, j))
    with cr.ConReg.from_problem(p, r_cap=8, precision=cr.CR_MIXED) as g:
        g.cr_set_factors(U, Z0, V)
        info = g.cr_project(1e-12)
        Zg = g.cr_get_factors()[1]
    Zo, _ = o.galerkin(U, V, tol=1e-14)
    assert info["iters"] > 0
    assert rel(Zg, Zo) < 1e-9


def test_mixed_greedy_invariants(cr, prob):
    p, o = prob
    r = 8
    Dn = np.linalg.norm(o.D())
    Js, rels = [], []
    with cr.ConReg.from_problem(p, r_cap=r, precision=cr.CR_MIXED) as g:
        for _ in range(r):
            g.cr_add_rank_one()
            g.cr_project(1e-12)
            res = g.cr_residual()
            U, Z, V = g.cr_get_factors()
            R = o.R_dense(U, Z, V)
            assert np.abs(U.T @ R @ V).max() <= 1e-9 * Dn
            assert abs(res["relres"] - np.linalg.norm(R) / Dn) <= 1e-8 * np.linalg.norm(R) / Dn
            Js.append(res["J"])
            rels.append(res["relres"])
    assert all(Js[k + 1] <= Js[k] * (1 + 1e-12) for k in range(r - 1))
    ref = o.greedy(r_max=r, tau=0.0, galerkin_tol=1e-13)
    assert rels[-1] <= 2.0 * ref.steps[-1].relres
