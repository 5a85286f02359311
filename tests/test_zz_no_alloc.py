"""The allocation-free entry point cr_solve_u_noalloc, for callers that cannot
allocate device memory, must give the same u-side solution as cr_solve_u.

It is called through the C ABI with device buffers the test owns (the CSR of
L_y, the data diagonal omega, the right side and the output) on two calls in a
row with different right sides, so a stale shared scratch array would show.
The problems span its launch shapes: 400 rows (one CTA), about 700 rows (a
2-CTA cluster) and a full 50^3 box of 125,000 rows (16 CTAs of 7,813 rows,
close to the 131,072-row limit of the static scratch).  This file is collected
last so that a run stopping at the first failure has already run every other
test; it also passes alone in a fresh process."""
import ctypes as C

import numpy as np
import pytest

from paper_1808_05510_gb300 import synth

pytestmark = pytest.mark.gpu

PROBLEMS = {"toy2d": synth.toy2d, "masked3d": synth.masked3d, "box50": synth.box3d}


@pytest.fixture(scope="module")
def lib():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1808_05510_gb300 import build

    build.build()
    from paper_1808_05510_gb300 import conreg as cr

    return cr, cr.load()


@pytest.mark.parametrize("name", list(PROBLEMS))
def test_noalloc_matches_cr_solve_u(lib, name):
    import torch

    cr, clib = lib
    p = PROBLEMS[name]()
    v = synth.random_unit(p.nx, 21)
    rng = np.random.default_rng(22)
    dev = torch.device("cuda", torch.cuda.current_device())
    stream = torch.cuda.current_stream()
    # coefficients of the u-side system for this v, evaluated on the host
    import scipy.sparse as sp

    Lx = sp.csr_matrix((p.Lx.val, p.Lx.col, p.Lx.rowptr), shape=(p.nx, p.nx))
    c = float(v @ (Lx @ v))
    d = float(np.linalg.norm(Lx @ v) ** 2)
    omega = p.Omega.astype(np.float64) @ ((p.X.T @ v) ** 2)
    rp = torch.tensor(p.Ly.rowptr, dtype=torch.int32, device=dev)
    co = torch.tensor(p.Ly.col, dtype=torch.int32, device=dev)
    va = torch.tensor(p.Ly.val, dtype=torch.float64, device=dev)
    om = torch.tensor(omega, dtype=torch.float64, device=dev)
    with cr.ConReg.from_problem(p, r_cap=1, pcg_tol=1e-13, pcg_maxit=50000) as g:
        for call in range(2):
            rhs = rng.standard_normal(p.ny)
            ref, _ = g.cr_solve_u(v, rhs)
            b = torch.tensor(rhs, dtype=torch.float64, device=dev)
            out = torch.full((p.ny,), float("nan"), dtype=torch.float64, device=dev)
            it = C.c_int32(-1)
            st = clib.cr_solve_u_noalloc(p.ny, rp.data_ptr(), co.data_ptr(), va.data_ptr(), p.lam, c, d,
                                         om.data_ptr(), b.data_ptr(), out.data_ptr(), 1e-13, 50000, C.byref(it),
                                         stream.cuda_stream)
            assert st == cr.CR_OK, clib.cr_last_error(None)
            assert it.value > 0
            got = out.cpu().numpy()
            err = np.linalg.norm(got - ref) / np.linalg.norm(ref)
            assert err < 1e-9, (name, call, err)
    # sizes beyond the static scratch are rejected with a clear error
    st = clib.cr_solve_u_noalloc(131073, rp.data_ptr(), co.data_ptr(), va.data_ptr(), p.lam, c, d, om.data_ptr(),
                                 om.data_ptr(), om.data_ptr(), 1e-10, 10, None, stream.cuda_stream)
    assert st == cr.CR_EINVAL and b"131072" in clib.cr_last_error(None)
