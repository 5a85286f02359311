"""cr_solve's automatic residual-check schedule (residual_every = 0): it stops on
a relative residual at or below the target, as the every-step schedule does, at
most two ranks later, with fewer residual checks.  Toy workload (20 x 20 grid,
5 injections, lambda = 100), which reaches relres 1e-6 near rank 88."""
import pytest

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


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_automatic_residual_schedule(cr, prec):
    p = synth.toy2d()
    precision = cr.CR_FP64 if prec == "fp64" else cr.CR_MIXED
    out = {}
    for every in (1, 0):
        with cr.ConReg.from_problem(p, r_cap=200, precision=precision, residual_every=every, profile=1) as g:
            info = g.cr_solve(200, 0.0, 1e-6)
            out[every] = (info, g.cr_get_stats()["phase_ms"]["resid"])
    (i1, c1), (i0, c0) = out[1], out[0]
    assert i1["stop_name"] == "relres" and i0["stop_name"] == "relres"
    assert i0["relres"] <= 1e-6
    assert i1["rank"] <= i0["rank"] <= i1["rank"] + 2, (i1["rank"], i0["rank"])
    assert c0 < 0.6 * c1, (c0, c1)
