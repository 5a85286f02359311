"""Host helpers of the learned preconditioner's training data on the CPU: the
Jacobi diagonals that scale the network's input equal the diagonals of the
oracle's own ALS operators (Eqs. ALS_linsys, ALS_linsys_v)."""
import numpy as np
import pytest

from oracle import Oracle
from paper_1808_05510_gb300 import learned, synth


@pytest.mark.parametrize("make", [synth.toy2d, synth.rect2d, synth.masked3d])
def test_jacobi_diagonals_match_the_oracle_operators(make):
    p = make()
    o = Oracle.from_problem(p)
    rng = np.random.default_rng(4)
    v = rng.standard_normal(p.nx)
    v /= np.linalg.norm(v)
    u = rng.standard_normal(p.ny)
    u /= np.linalg.norm(u)
    dA = np.asarray(o.A_hat(v).diagonal())
    assert np.allclose(learned.jacobi_diag(p, v), dA, rtol=1e-13, atol=0)
    S, s = o.B_hat(u)
    X = p.X.toarray() if hasattr(p.X, "toarray") else np.asarray(p.X)
    B = S.toarray() + (X * s) @ X.T  # the dense B_hat
    assert np.allclose(learned.jacobi_diag_v(p, u), np.diag(B), rtol=1e-13, atol=0)


def test_box_mask_is_three_dimensional():
    g = synth.toy2d().grid_x
    m = learned.box_mask(g)
    assert m.ndim == 3 and m.shape[:2] == g.mask.shape and m.sum() == g.n
