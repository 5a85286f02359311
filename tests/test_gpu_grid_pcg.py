"""The grid-wide PCG (vectors in HBM, every SM) against the float64 oracle:
on a 180,000-voxel box, beyond one thread-block cluster's shared memory (the
library switches to it by itself), in the float64 form and in the mixed form
(float32 grid kernel under float64 refinement), both ALS sides; and a greedy
trajectory with the grid kernel forced on a small problem."""
import numpy as np
import pytest

from oracle import Oracle
from paper_1808_05510_gb300 import synth

pytestmark = pytest.mark.gpu


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
def big():
    rng = np.random.default_rng(41)
    g = synth.Grid(np.ones((50, 60, 60), dtype=bool))
    L = synth.grid_laplacian(g)
    X = synth.gaussian_injections(g, 4, rng, 2.0, 3.0, 1.0, 1.0)
    Om = (X <= 0.4).astype(np.uint8)
    Y = rng.standard_normal((g.n, 4)) * Om
    p = synth.Problem("box180k", g, g, L, L, X, Y, Om, 1.0, 4)
    return p, Oracle(L, L, X, Y, Om, 1.0)


def rel(a, b):
    return np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(b), 1e-300)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_grid_pcg_beyond_one_cluster(cr, big, prec):
    p, o = big
    assert p.nx == 180000
    rng = np.random.default_rng(42)
    v = p.X.sum(axis=1)
    v /= np.linalg.norm(v)
    u = rng.standard_normal(p.ny)
    u /= np.linalg.norm(u)
    rhs_u = rng.standard_normal(p.ny)
    rhs_v = rng.standard_normal(p.nx)
    precision = cr.CR_FP64 if prec == "fp64" else cr.CR_MIXED
    with cr.ConReg.from_problem(p, r_cap=2, pcg_tol=1e-12, pcg_maxit=100000, precision=precision) as g:
        uh, itu = g.cr_solve_u(v, rhs_u)
        vh, itv = g.cr_solve_v(u, rhs_v)
    assert itu > 0 and itv > 0
    assert rel(uh, o.solve_u(v, rhs_u)) < 1e-9
    assert rel(vh, o.solve_v(u, rhs_v)) < 1e-9


def test_greedy_trajectory_grid_kernel(cr):
    p = synth.masked3d()
    o = Oracle.from_problem(p)
    r = 5
    steps = []
    with cr.ConReg.from_problem(p, r_cap=r, pcg_tol=1e-13, pcg_maxit=50000, als_sweeps=2, pcg_kernel=2) as g:
        for _ in range(r):
            g.cr_add_rank_one()
            g.cr_project(1e-13)
            U, Z, V = g.cr_get_factors()
            steps.append(U @ Z @ V.T)
    ref = []
    o.greedy(r_max=r, tau=0.0, als_sweeps=2, galerkin_tol=1e-14,
             callback=lambda st, U, Z, V: ref.append(U @ Z @ V.T))
    for Wg, Wo in zip(steps, ref):
        assert rel(Wg, Wo) < 1e-9
