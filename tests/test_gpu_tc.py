"""Tensor-core (tcgen05, BF16 hi/lo operands, float32 accumulation) Galerkin
assembly G_a = U^T diag(Omega_a) U against the float64 oracle.

Stated error: each BF16 hi/lo pair carries U to ~2^-17 relative and the
dropped lo*lo product is ~2^-16 relative, so G_a agrees with float64 to
5e-5 in the Frobenius norm (the float32 rounding of the float64 path to 1e-6).
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


@pytest.mark.parametrize("name,j", [("toy2d", 6), ("toy2d9", 20), ("masked3d", 40), ("masked3d", 100),
                                    ("masked3d", 128), ("visual", 64)])
def test_tensor_core_assembly(cr, name, j):
    p = {"toy2d": lambda: synth.toy2d(), "toy2d9": lambda: synth.toy2d(m=9),
         "masked3d": lambda: synth.masked3d(), "visual": lambda: synth.visual_cortex()}[name]()
    o = Oracle.from_problem(p)
    rng = np.random.default_rng(40 + j)
    U, _ = np.linalg.qr(rng.standard_normal((p.ny, j)))
    V, _ = np.linalg.qr(rng.standard_normal((p.nx, j)))
    Z = rng.standard_normal((j, j))
    with cr.ConReg.from_problem(p, r_cap=j, precision=cr.CR_MIXED) as g:
        g.cr_set_factors(U, Z, V)
        Gt = g.cr_galerkin_assembly(0)
        Gf = g.cr_galerkin_assembly(1)
    for a in range(p.m):
        ref = U.T @ (p.Omega[:, a][:, None] * U)
        assert np.linalg.norm(Gt[a] - ref) <= 5e-5 * np.linalg.norm(ref), a
        assert np.linalg.norm(Gf[a] - ref) <= 1e-6 * np.linalg.norm(ref), a
