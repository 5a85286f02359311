"""GPU parity of the multigrid-preconditioned ALS sub-solves (Eqs. ALS_linsys and
ALS_linsys_v, Sec. 2.3; cr_options.precond = CR_PRECOND_MULTIGRID).

The preconditioner changes how the systems are solved, not what is solved, so
the bar is the same as for Jacobi-PCG: solutions within 1e-9 of the oracle's
(its dense Cholesky or CG to 1e-14; the GPU solves to 1e-13), greedy
trajectories within 1e-9, and a normwise backward error of the GPU solution,
|A x - b| / (|A|_F |x| + |b|) measured in float64 by the oracle, below 1e-13.
Where the system's condition number (dense, for n <= 2000) makes 1e-9
unattainable for any float64 solver at these tolerances -- the 1-D chain's
v-side system with a smooth u has cond 3.7e6, and numpy's dense solve of it
leaves a relative residual of 1.7e-11 -- the solution bar is
20 cond (1e-13 + 1e-14) instead.  Beside parity: the preconditioner must cut the
iterations of the smooth (ill-conditioned) sub-systems by a wide margin, the
solves must repeat bit for bit, and a problem too small for a hierarchy falls
back to Jacobi."""
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


PROBLEMS = {"paper_toy": synth.paper_toy, "toy2d": synth.toy2d, "masked3d": synth.masked3d,
            "visual": synth.visual_cortex}


@pytest.fixture(scope="module", params=list(PROBLEMS))
def prob(request):
    p = PROBLEMS[request.param]()
    return request.param, p, Oracle.from_problem(p)


def rel(a, b):
    return np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(b), 1e-300)


def b_apply(o, p, u, x):
    S, s = o.B_hat(u)
    return S @ x + p.X @ (s * (p.X.T @ x))


def check_solve(apply, fro, dense, x, b, x_ref):
    """Backward error <= 1e-13 and the solution within the conditioning bar of the oracle's."""
    eta = np.linalg.norm(apply(x) - b) / (fro * np.linalg.norm(x) + np.linalg.norm(b))
    assert eta <= 1e-13, eta
    bar = 1e-9
    if dense is not None:
        bar = max(bar, 20.0 * np.linalg.cond(dense) * 1.1e-13)
    assert rel(x, x_ref) < bar, (rel(x, x_ref), bar)


def solves(cr, p, v, u, rhs_u, rhs_v, prec, precond, **kw):
    precision = cr.CR_FP64 if prec == "fp64" else cr.CR_MIXED
    with cr.ConReg.from_problem(p, r_cap=4, pcg_tol=1e-13, pcg_maxit=200000, precision=precision, precond=precond,
                                **kw) as g:
        uh, itu = g.cr_solve_u(v, rhs_u)
        vh, itv = g.cr_solve_v(u, rhs_v)
        st = g.cr_get_stats()
    return uh, vh, itu, itv, st


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_multigrid_subsolves_match_oracle(cr, prob, prec):
    name, p, o = prob
    v = synth.smooth_unit(p.grid_x, 81)
    u = synth.smooth_unit(p.grid_y, 82)
    rng = np.random.default_rng(83)
    rhs_u = rng.standard_normal(p.ny)
    rhs_v = rng.standard_normal(p.nx)
    uh, vh, itu, itv, st = solves(cr, p, v, u, rhs_u, rhs_v, prec, cr.CR_PRECOND_MULTIGRID)
    assert min(st["pcg_multigrid"]) >= 2, st
    import scipy.sparse.linalg as spla

    Ah = o.A_hat(v)
    S, s = o.B_hat(u)
    lowrank = (p.X * s) @ p.X.T if p.nx <= 2000 else None
    Bd = S.toarray() + lowrank if lowrank is not None else None
    b_fro = spla.norm(S) + float(np.sqrt(np.sum(((p.X.T @ p.X) * np.outer(s, s)) * (p.X.T @ p.X))))
    check_solve(lambda x: Ah @ x, spla.norm(Ah), Ah.toarray() if p.ny <= 2000 else None, uh, rhs_u,
                o.solve_u(v, rhs_u))
    check_solve(lambda x: b_apply(o, p, u, x), b_fro, Bd, vh, rhs_v, o.solve_v(u, rhs_v))
    if prec == "fp64":
        _, _, ju, jv, _ = solves(cr, p, v, u, rhs_u, rhs_v, prec, cr.CR_PRECOND_JACOBI)
        # the smooth sub-systems: multigrid needs a fraction of Jacobi's iterations
        assert 3 * itu < ju and 3 * itv < jv, (name, itu, ju, itv, jv)


def test_multigrid_repeats_bit_for_bit(cr):
    p = synth.visual_cortex()
    v = synth.smooth_unit(p.grid_x, 91)
    rhs = np.random.default_rng(92).standard_normal(p.ny)
    outs = []
    for _ in range(2):
        with cr.ConReg.from_problem(p, r_cap=2, precond=cr.CR_PRECOND_MULTIGRID) as g:
            outs.append(g.cr_solve_u(v, rhs))
    assert np.array_equal(outs[0][0], outs[1][0]) and outs[0][1] == outs[1][1]


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("name", ["masked3d", "visual"])
def test_multigrid_greedy_trajectory(cr, prec, name):
    p = PROBLEMS[name]()
    o = Oracle.from_problem(p)
    r = 4
    precision = cr.CR_FP64 if prec == "fp64" else cr.CR_MIXED
    Ws = []
    with cr.ConReg.from_problem(p, r_cap=r, pcg_tol=1e-13, pcg_maxit=200000, als_sweeps=2, precision=precision,
                                precond=cr.CR_PRECOND_MULTIGRID) as g:
        for _ in range(r):
            g.cr_add_rank_one()
            g.cr_project(1e-13)
            Ws.append(g.cr_get_factors())
    ref = []
    o.greedy(r_max=r, tau=0.0, als_sweeps=2, galerkin_tol=1e-14, dense_residual=False,
             callback=lambda st, U, Z, V: ref.append((U.copy(), Z.copy(), V.copy())))
    for (Ug, Zg, Vg), (Uo, Zo, Vo) in zip(Ws, ref):
        Qu, Ru = np.linalg.qr(np.hstack([Ug, Uo]))
        Qv, Rv = np.linalg.qr(np.hstack([Vg, Vo]))
        j = Zg.shape[0]
        M = np.zeros((2 * j, 2 * j))
        M[:j, :j] = Zg
        M[j:, j:] = -Zo
        diff = np.linalg.norm(Ru @ M @ Rv.T) / np.linalg.norm(Zo)  # |W_gpu - W_oracle| / |W_oracle|
        assert diff < 1e-9, diff


@pytest.mark.parametrize("cs", [8, 16])
def test_multigrid_forced_cluster_sizes(cr, cs):
    p = synth.masked3d()
    o = Oracle.from_problem(p)
    v = synth.smooth_unit(p.grid_x, 95)
    u = synth.smooth_unit(p.grid_y, 96)
    rng = np.random.default_rng(97)
    rhs_u = rng.standard_normal(p.ny)
    rhs_v = rng.standard_normal(p.nx)
    uh, vh, _, _, st = solves(cr, p, v, u, rhs_u, rhs_v, "fp64", cr.CR_PRECOND_MULTIGRID, cluster_size=cs)
    assert st["pcg_cluster"] == [cs, cs] and min(st["pcg_multigrid"]) >= 2
    assert rel(uh, o.solve_u(v, rhs_u)) < 1e-9
    assert rel(vh, o.solve_v(u, rhs_v)) < 1e-9


def test_too_small_for_a_hierarchy_falls_back_to_jacobi(cr):
    p = synth.rect2d()  # 63 and 48 rows: no coarsening below the dense size
    o = Oracle.from_problem(p)
    v = synth.random_unit(p.nx, 98)
    rhs = np.random.default_rng(99).standard_normal(p.ny)
    with cr.ConReg.from_problem(p, r_cap=4, pcg_tol=1e-13, precond=cr.CR_PRECOND_MULTIGRID) as g:
        uh, _ = g.cr_solve_u(v, rhs)
        assert g.cr_get_stats()["pcg_multigrid"] == [0, 0]
    assert rel(uh, o.solve_u(v, rhs)) < 1e-9


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("lam", [1e2, 2e3])
def test_auto_choice_per_side(cr, prec, lam):
    """CR_PRECOND_AUTO: multigrid in the float64 form; in the mixed form Jacobi at
    this size for lambda < 1e3 and multigrid from 1e3 on.  Either way the solves
    meet the oracle's."""
    import dataclasses

    p = dataclasses.replace(synth.visual_cortex(), lam=lam)
    o = Oracle.from_problem(p)
    v = synth.smooth_unit(p.grid_x, 101)
    u = synth.smooth_unit(p.grid_y, 102)
    rng = np.random.default_rng(103)
    rhs_u = rng.standard_normal(p.ny)
    rhs_v = rng.standard_normal(p.nx)
    uh, vh, _, _, st = solves(cr, p, v, u, rhs_u, rhs_v, prec, cr.CR_PRECOND_AUTO)
    mg = prec == "fp64" or lam >= 1e3
    assert st["pcg_multigrid"] == ([3, 3] if mg else [0, 0]), st["pcg_multigrid"]
    tol = 1e-9 if lam < 1e3 else 1e-8
    assert rel(uh, o.solve_u(v, rhs_u)) < tol
    assert rel(vh, o.solve_v(u, rhs_v)) < tol
