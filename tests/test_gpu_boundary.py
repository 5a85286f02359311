"""GPU round trips of the boundary's input and checkpoint calls (Algorithm 1's
input and output lines): a problem created from device buffers
(mem_kind = CR_MEM_DEVICE) runs exactly like one created from host buffers; a
checkpoint taken with cr_get_state and restored with cr_set_state into a fresh
problem continues the greedy run bit for bit; voxel grids given at creation are
those of cr_set_voxel_grid."""
import ctypes as C

import numpy as np
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
def test_device_inputs_match_host_inputs(cr, prec):
    p = synth.masked3d()
    precision = cr.CR_FP64 if prec == "fp64" else cr.CR_MIXED
    out = []
    for dev in (False, True):
        with cr.ConReg.from_problem(p, r_cap=5, als_sweeps=2, precision=precision, device_inputs=dev) as g:
            g.cr_solve(5, 0.0, 0.0)
            out.append(g.cr_get_factors())
    for a, b in zip(out[0], out[1]):
        assert np.array_equal(a, b)


def test_device_kind_with_host_pointers_is_rejected(cr):
    p = synth.rect2d()
    lib = cr.load()
    g = cr.ConReg.from_problem(p, r_cap=2)  # builds a host descriptor; reuse its arrays
    g.close()
    keep = []
    d = cr.cr_problem_desc()
    d.nx, d.ny, d.ninj = p.nx, p.ny, p.m
    for name, L in (("Lx", p.Lx), ("Ly", p.Ly)):
        rp, co, va = (np.ascontiguousarray(L.rowptr, np.int32), np.ascontiguousarray(L.col, np.int32),
                      np.ascontiguousarray(L.val, np.float64))
        keep += [rp, co, va]
        setattr(d, name, cr.cr_csr(L.n, cr._ptr(rp, cr._ip), cr._ptr(co, cr._ip), cr._ptr(va)))
    X, Y, Om = (np.asfortranarray(p.X), np.asfortranarray(p.Y), np.asfortranarray(p.Omega.astype(np.uint8)))
    keep += [X, Y, Om]
    d.X_host, d.ldx = cr._ptr(X), p.nx
    d.Y_host, d.ldy = cr._ptr(Y), p.ny
    d.Omega_host, d.ldo = cr._ptr(Om, cr._up), p.ny
    d.lambda_ = p.lam
    d.mem_kind = cr.CR_MEM_DEVICE
    h = C.c_void_p()
    opts = cr.default_options(r_cap=2)
    assert lib.cr_create(C.byref(d), C.byref(opts), C.byref(h)) == cr.CR_EINVAL
    assert not h.value and b"device memory" in lib.cr_last_error(None)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_checkpoint_continues_bit_for_bit(cr, prec):
    p = synth.masked3d()
    precision = cr.CR_FP64 if prec == "fp64" else cr.CR_MIXED
    kw = dict(r_cap=9, precision=precision, precond=cr.CR_PRECOND_MULTIGRID)
    with cr.ConReg.from_problem(p, **kw) as g:
        g.cr_solve(5, 0.0, 0.0)
        state = g.cr_get_state()
        dW5 = g.cr_residual(relres=False, J=False)["dW"]
        g.cr_solve(8, 0.0, 0.0)
        ref = g.cr_get_factors()
        ref_res = g.cr_residual()
    with cr.ConReg.from_problem(p, **kw) as g:
        g.cr_set_state(state)
        assert g.cr_get_rank() == 5
        assert g.cr_residual(relres=False, J=False)["dW"] == dW5
        g.cr_solve(8, 0.0, 0.0)
        got = g.cr_get_factors()
        got_res = g.cr_residual()
    for a, b in zip(ref, got):
        assert np.array_equal(a, b)
    assert got_res == ref_res


def test_checkpoint_rejects_foreign_and_corrupt_states(cr):
    import dataclasses

    p = synth.masked3d()
    with cr.ConReg.from_problem(p, r_cap=6) as g:
        g.cr_solve(4, 0.0, 0.0)
        state = g.cr_get_state()
    bad = bytearray(state)
    bad[-3] ^= 0x40  # one flipped bit in V
    with cr.ConReg.from_problem(p, r_cap=6) as g:
        with pytest.raises(cr.ConRegError) as e:
            g.cr_set_state(bytes(bad))
        assert e.value.status == cr.CR_EINVAL
        with pytest.raises(cr.ConRegError) as e:
            g.cr_set_state(state[:100])
        assert e.value.status == cr.CR_EINVAL
    with cr.ConReg.from_problem(dataclasses.replace(p, lam=2 * p.lam), r_cap=6) as g:
        with pytest.raises(cr.ConRegError) as e:
            g.cr_set_state(state)
        assert e.value.status == cr.CR_EINVAL
    with cr.ConReg.from_problem(p, r_cap=3) as g:
        with pytest.raises(cr.ConRegError) as e:
            g.cr_set_state(state)
        assert e.value.status == cr.CR_ESTATE


def test_grids_at_creation_equal_set_voxel_grid(cr):
    """The learned preconditioner needs the voxel boxes; given at creation they
    act exactly as cr_set_voxel_grid afterwards (same learned solve, bit for bit)."""
    p = synth.toy2d()
    net = cr.ConvNet(p.grid_y.mask.shape, batch_cap=1, seed=11)
    rng = np.random.default_rng(12)
    net.set_params((0.05 * rng.standard_normal(cr.ConvNet.param_count())).astype(np.float32))
    v = synth.smooth_unit(p.grid_x, 13)
    rhs = rng.standard_normal(p.ny)
    outs = []
    for at_create in (True, False):
        kw = dict(r_cap=2, precond=cr.CR_PRECOND_LEARNED, learned_judge=1)
        if at_create:
            g = cr.ConReg.from_problem(p, grids=(p.grid_x.mask, p.grid_y.mask), **kw)
        else:
            g = cr.ConReg.from_problem(p, **kw)
            g.cr_set_voxel_grid(0, p.grid_y.mask)
            g.cr_set_voxel_grid(1, p.grid_x.mask)
        with g:
            g.cr_set_preconditioner(net)
            g.cr_solve_u(v, rhs)  # the judge's Jacobi solve
            outs.append(g.cr_solve_u(v, rhs))  # learned (flexible CG)
            st = g.cr_get_stats()
            assert st["learned_solves"] + st["learned_fallbacks"] >= 1
    net.close()
    assert np.array_equal(outs[0][0], outs[1][0]) and outs[0][1] == outs[1][1]
