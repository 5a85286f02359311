"""Thin Python binding of the libconreg C ABI (``include/conreg.h``).

Argument marshalling only: every numerical step runs in the CUDA library.  The
functions keep the C names (``cr_create``, ``cr_add_rank_one``, ...); the
``ConReg`` class wraps a problem handle.  PyTorch supplies device memory (its
caching allocator is passed as the library's allocator hook) and the CUDA
stream.  There is no CPU fallback: without the built library or a GPU every
call raises.
"""
from __future__ import annotations

import ctypes as C
import os
from typing import Optional

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_PKG, "libconreg.so")
_lib = None

CR_OK, CR_EINVAL, CR_ENOMEM, CR_ECUDA, CR_ENOTCONV, CR_ETIMEOUT, CR_ERANK, CR_ESTATE = range(8)
CR_FP64, CR_MIXED = 0, 1
CR_PRECOND_JACOBI, CR_PRECOND_LEARNED, CR_PRECOND_MULTIGRID, CR_PRECOND_AUTO = 0, 1, 2, 3
CR_GALERKIN_AUTO, CR_GALERKIN_JACOBI, CR_GALERKIN_EIGEN = 0, 1, 2
STOP_NAMES = {0: "none", 1: "r_max", 2: "dW", 3: "relres", 4: "rank"}

_dp = C.POINTER(C.c_double)
_ip = C.POINTER(C.c_int32)
_up = C.POINTER(C.c_uint8)


class cr_csr(C.Structure):
    _fields_ = [("n", C.c_int64), ("rowptr", _ip), ("col", _ip), ("val", _dp)]


class cr_grid(C.Structure):
    _fields_ = [("dims", C.c_int32 * 3), ("box_index", _ip)]


CR_MEM_HOST, CR_MEM_DEVICE = 0, 1


class cr_problem_desc(C.Structure):
    _fields_ = [("nx", C.c_int64), ("ny", C.c_int64), ("ninj", C.c_int64), ("Lx", cr_csr), ("Ly", cr_csr),
                ("X_host", _dp), ("ldx", C.c_int64), ("Y_host", _dp), ("ldy", C.c_int64),
                ("Omega_host", _up), ("ldo", C.c_int64), ("lambda_", C.c_double), ("mem_kind", C.c_int32),
                ("grid_x", cr_grid), ("grid_y", cr_grid)]


ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p)
FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_size_t, C.c_void_p)


class cr_options(C.Structure):
    _fields_ = [("struct_size", C.c_size_t), ("r_cap", C.c_int32), ("precision", C.c_int32),
                ("precond", C.c_int32), ("pcg_tol", C.c_double), ("pcg_maxit", C.c_int32),
                ("als_delta", C.c_double), ("als_max_iter", C.c_int32), ("als_sweeps", C.c_int32),
                ("galerkin_maxit", C.c_int32), ("residual_every", C.c_int32), ("cluster_size", C.c_int32),
                ("profile", C.c_int32), ("pcg_kernel", C.c_int32), ("galerkin_kernel", C.c_int32),
                ("seed", C.c_uint64), ("stream", C.c_void_p), ("alloc", ALLOC_FN), ("free", FREE_FN),
                ("alloc_ctx", C.c_void_p), ("galerkin_ctas", C.c_int32), ("learned_judge", C.c_int32),
                ("galerkin_form", C.c_int32)]


class cr_rank1_info(C.Structure):
    _fields_ = [("rank", C.c_int32), ("sweeps", C.c_int32), ("delta", C.c_double), ("unorm", C.c_double),
                ("vnorm", C.c_double), ("pcg_iters_u", C.c_int32), ("pcg_iters_v", C.c_int32),
                ("pcg_relres_max", C.c_double)]


class cr_proj_info(C.Structure):
    _fields_ = [("iters", C.c_int32), ("relres", C.c_double)]


PHASES = ["pcg_u", "pcg_v", "rhs", "orth", "galerkin", "resid", "pcg_kernel", "basis", "pcg_kernel_v", "p9"]


class cr_stats(C.Structure):
    _fields_ = [("launches", C.c_int64), ("pcg_solves", C.c_int64), ("pcg_iters", C.c_int64),
                ("h2d_bytes", C.c_int64), ("d2h_bytes", C.c_int64), ("phase_ms", C.c_double * 10), ("phase_calls", C.c_int64 * 10),
                ("learned_solves", C.c_int64), ("learned_fallbacks", C.c_int64), ("learned_off", C.c_int64),
                ("mixed_handovers", C.c_int64), ("pcg_cluster", C.c_int64 * 2),
                ("pcg_multigrid", C.c_int64 * 2), ("galerkin_eigen", C.c_int64 * 2),
                ("pcg_iters_side", C.c_int64 * 2), ("pcg_bytes_per_iter", C.c_double * 2)]


class cr_solve_info(C.Structure):
    _fields_ = [("rank", C.c_int32), ("stop", C.c_int32), ("relres", C.c_double), ("dW", C.c_double),
                ("J", C.c_double), ("pcg_iters", C.c_int64), ("cg_iters", C.c_int64), ("seconds", C.c_double)]


class cr_member(C.Structure):
    _fields_ = [("lambda_", C.c_double), ("fit_cols", _ip), ("n_fit", C.c_int32), ("test_cols", _ip),
                ("n_test", C.c_int32)]


class cr_member_result(C.Structure):
    _fields_ = [("status", C.c_int32), ("rank", C.c_int32), ("stop", C.c_int32), ("slot", C.c_int32),
                ("relres", C.c_double), ("dW", C.c_double), ("J", C.c_double), ("cv_num", C.c_double),
                ("cv_den", C.c_double), ("pcg_iters", C.c_int64), ("cg_iters", C.c_int64), ("seconds", C.c_double)]


class cr_solution_stats(C.Structure):
    _fields_ = [("entries", C.c_int64), ("n_negative", C.c_int64), ("w_min", C.c_double), ("w_max", C.c_double),
                ("w_fro2", C.c_double), ("neg_fro2", C.c_double), ("ref_fro2", C.c_double),
                ("diff_fro2", C.c_double), ("diff_maxabs", C.c_double), ("rms", C.c_double), ("rel", C.c_double)]


# Every exported symbol with its (restype, argtypes); include/conreg.h declares the same set.
SIGNATURES = {
    "cr_options_default": (C.c_int, [C.POINTER(cr_options)]),
    "cr_lambda_from_bar": (C.c_double, [C.c_double, C.c_int64, C.c_int64]),
    "cr_create": (C.c_int, [C.POINTER(cr_problem_desc), C.POINTER(cr_options), C.POINTER(C.c_void_p)]),
    "cr_destroy": (None, [C.c_void_p]),
    "cr_add_rank_one": (C.c_int, [C.c_void_p, C.POINTER(cr_rank1_info)]),
    "cr_project": (C.c_int, [C.c_void_p, C.c_double, C.POINTER(cr_proj_info)]),
    "cr_residual": (C.c_int, [C.c_void_p, _dp, _dp, _dp]),
    "cr_solve": (C.c_int, [C.c_void_p, C.c_int32, C.c_double, C.c_double, C.POINTER(cr_solve_info)]),
    "cr_get_rank": (C.c_int, [C.c_void_p, _ip]),
    "cr_get_factors": (C.c_int, [C.c_void_p, _dp, C.c_int64, _dp, C.c_int64, _dp, C.c_int64]),
    "cr_set_factors": (C.c_int, [C.c_void_p, C.c_int32, _dp, C.c_int64, _dp, C.c_int64, _dp, C.c_int64]),
    "cr_get_state": (C.c_int, [C.c_void_p, C.c_void_p, C.POINTER(C.c_size_t)]),
    "cr_set_state": (C.c_int, [C.c_void_p, C.c_void_p, C.c_size_t]),
    "cr_apply_residual": (C.c_int, [C.c_void_p, C.c_int32, _dp, _dp]),
    "cr_solve_u": (C.c_int, [C.c_void_p, _dp, _dp, _dp, _ip]),
    "cr_solve_v": (C.c_int, [C.c_void_p, _dp, _dp, _dp, _ip]),
    "cr_get_stats": (C.c_int, [C.c_void_p, C.POINTER(cr_stats), C.c_int32]),
    "cr_galerkin_assembly": (C.c_int, [C.c_void_p, C.c_int32, C.POINTER(C.c_float), C.c_int64]),
    "cr_net_param_count": (C.c_int64, []),
    "cr_net_create": (C.c_int, [C.c_int32, C.c_int32, C.c_int32, C.c_int32, C.c_uint64, C.c_void_p,
                                C.POINTER(C.c_void_p)]),
    "cr_net_destroy": (None, [C.c_void_p]),
    "cr_net_get_params": (C.c_int, [C.c_void_p, C.POINTER(C.c_float), C.c_int64]),
    "cr_net_set_params": (C.c_int, [C.c_void_p, C.POINTER(C.c_float), C.c_int64]),
    "cr_net_forward": (C.c_int, [C.c_void_p, C.c_int32, C.c_void_p, C.c_void_p]),
    "cr_net_gradients": (C.c_int, [C.c_void_p, C.c_int32, C.c_void_p, C.c_void_p, C.c_void_p,
                                   C.POINTER(C.c_float), C.POINTER(C.c_float)]),
    "cr_net_train_step": (C.c_int, [C.c_void_p, C.c_int32, C.c_void_p, C.c_void_p, C.c_void_p, C.c_float,
                                    C.POINTER(C.c_float)]),
    "cr_arrow_check": (C.c_int, [C.c_int32, _dp, _dp, C.c_double, _dp, _dp]),
    "cr_net_check_f64": (C.c_int, [C.c_int32, C.c_int32, C.c_int32, C.c_int32, _dp, _dp, _dp, _up, _dp, _dp, _dp]),
    "cr_set_voxel_grid": (C.c_int, [C.c_void_p, C.c_int32, _ip, _ip]),
    "cr_set_preconditioner": (C.c_int, [C.c_void_p, C.c_void_p]),
    "cr_solve_u_noalloc": (C.c_int, [C.c_int64, C.c_void_p, C.c_void_p, C.c_void_p, C.c_double, C.c_double,
                                     C.c_double, C.c_void_p, C.c_void_p, C.c_void_p, C.c_double, C.c_int32, _ip,
                                     C.c_void_p]),
    "cr_cv_error": (C.c_int, [C.c_void_p, C.c_int32, _dp, C.c_int64, _dp, C.c_int64, _up, C.c_int64, _dp, _dp]),
    "cr_svd_factors": (C.c_int, [C.c_void_p, _dp, C.c_int64, _dp, _dp, C.c_int64]),
    "cr_solution_report": (C.c_int, [C.c_void_p, C.c_int32, C.c_int32, _dp, C.c_int64, _dp, C.c_int64, _dp, C.c_int64,
                                     _dp, C.c_int64, C.POINTER(cr_solution_stats)]),
    "cr_solve_batch": (C.c_int, [C.POINTER(cr_problem_desc), C.POINTER(cr_options), C.POINTER(cr_member), C.c_int32,
                                 C.c_int32, C.c_double, C.c_double, C.c_int32, C.POINTER(cr_member_result),
                                 C.POINTER(C.c_void_p)]),
    "cr_status_str": (C.c_char_p, [C.c_int]),
    "cr_last_error": (C.c_char_p, [C.c_void_p]),
}


class ConRegError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{msg} (status {status})")
        self.status = status


def lib_path() -> str:
    return _LIB_PATH


def load():
    """Load libconreg.so (built by ``paper_1808_05510_gb300.build``); raises if missing."""
    global _lib
    if _lib is None:
        if not os.path.exists(_LIB_PATH):
            raise RuntimeError("libconreg.so is not built: run `python -c 'import __graft_entry__ as g; g.build()'`")
        lib = C.CDLL(_LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
    return _lib


def _ptr(a: np.ndarray, t=_dp):
    return a.ctypes.data_as(t)


def _check(st: int, handle=None, where: str = ""):
    if st != CR_OK:
        lib = load()
        msg = lib.cr_last_error(handle).decode() if lib.cr_last_error(handle) else ""
        raise ConRegError(st, f"{where}: {lib.cr_status_str(st).decode()}: {msg}")


def _f64(a) -> np.ndarray:
    return np.asfortranarray(np.asarray(a, dtype=np.float64))


class _TorchAllocator:
    """Routes the library's device allocations through torch's caching allocator."""

    def __init__(self, stream_ptr: int):
        import torch

        self._torch = torch
        self._stream = stream_ptr
        self._alloc = ALLOC_FN(self._do_alloc)
        self._free = FREE_FN(self._do_free)

    def _do_alloc(self, nbytes, ctx):
        try:
            return int(self._torch.cuda.caching_allocator_alloc(int(nbytes), stream=self._stream))
        except Exception:  # out of memory -> the library reports CR_ENOMEM
            return None

    def _do_free(self, ptr, nbytes, ctx):
        self._torch.cuda.caching_allocator_delete(ptr)


def default_options(**kw) -> cr_options:
    o = cr_options()
    _check(load().cr_options_default(C.byref(o)), None, "cr_options_default")
    for k, v in kw.items():
        if not hasattr(o, k):
            raise TypeError(f"unknown option {k}")
        setattr(o, k, v)
    return o


class ConReg:
    """One problem instance on the current CUDA device (see ``include/conreg.h``)."""

    def __init__(self, Lx, Ly, X, Y, Omega, lam: float, stream=None, use_torch_allocator: bool = True,
                 device_inputs: bool = False, grids=None, **opts):
        """``device_inputs``: hand the library device copies of every array
        (mem_kind = CR_MEM_DEVICE) instead of host pointers.  ``grids``: optional
        (mask_x, mask_y) voxel boxes (C-order masks, rows numbered in that order)
        passed at creation."""
        import torch

        if not torch.cuda.is_available():
            raise RuntimeError("ConReg needs a CUDA device")
        lib = load()
        self._lib = lib
        self._keep = []
        self.X = _f64(X)
        self.Y = _f64(Y)
        self.Om = np.asfortranarray(np.asarray(Omega, dtype=np.uint8))
        self.nx, self.m = self.X.shape
        self.ny = self.Y.shape[0]
        d = cr_problem_desc()
        d.nx, d.ny, d.ninj = self.nx, self.ny, self.m
        for name, L in (("Lx", Lx), ("Ly", Ly)):
            rp = np.ascontiguousarray(L.rowptr, dtype=np.int32)
            co = np.ascontiguousarray(L.col, dtype=np.int32)
            va = np.ascontiguousarray(L.val, dtype=np.float64)
            self._keep += [rp, co, va]
            setattr(d, name, cr_csr(L.n, _ptr(rp, _ip), _ptr(co, _ip), _ptr(va)))
        d.X_host, d.ldx = _ptr(self.X), self.nx
        d.Y_host, d.ldy = _ptr(self.Y), self.ny
        d.Omega_host, d.ldo = _ptr(self.Om, _up), self.ny
        d.lambda_ = float(lam)
        if grids is not None:
            for name, mask in (("grid_x", grids[0]), ("grid_y", grids[1])):
                if mask is None:
                    continue
                dims = list(mask.shape) + [1] * (3 - mask.ndim)
                idx = np.ascontiguousarray(np.flatnonzero(np.asarray(mask).ravel()), dtype=np.int32)
                self._keep.append(idx)
                g = getattr(d, name)
                g.dims[:] = dims
                g.box_index = _ptr(idx, _ip)
        if device_inputs:
            # device copies of every array, the descriptor pointing at them
            dev = torch.device("cuda", torch.cuda.current_device())

            def on_dev(a):
                t = torch.from_numpy(np.array(a, copy=True, order="F").ravel(order="F")).to(dev)
                self._keep.append(t)
                return t.data_ptr()

            for name in ("Lx", "Ly"):
                c = getattr(d, name)
                L = Lx if name == "Lx" else Ly
                setattr(d, name, cr_csr(L.n, C.cast(C.c_void_p(on_dev(np.asarray(L.rowptr, np.int32))), _ip),
                                        C.cast(C.c_void_p(on_dev(np.asarray(L.col, np.int32))), _ip),
                                        C.cast(C.c_void_p(on_dev(np.asarray(L.val, np.float64))), _dp)))
            d.X_host = C.cast(C.c_void_p(on_dev(self.X)), _dp)
            d.Y_host = C.cast(C.c_void_p(on_dev(self.Y)), _dp)
            d.Omega_host = C.cast(C.c_void_p(on_dev(self.Om)), _up)
            for name in ("grid_x", "grid_y"):
                g = getattr(d, name)
                if g.box_index:
                    n = self.nx if name == "grid_x" else self.ny
                    host = np.ctypeslib.as_array(g.box_index, shape=(n,)).copy()
                    g.box_index = C.cast(C.c_void_p(on_dev(host)), _ip)
            d.mem_kind = CR_MEM_DEVICE
            torch.cuda.synchronize()
        if stream is None:
            stream = torch.cuda.current_stream()
        self.stream = stream
        o = default_options(**opts)
        o.stream = C.c_void_p(stream.cuda_stream)
        self._allocator = None
        if use_torch_allocator:
            self._allocator = _TorchAllocator(stream.cuda_stream)
            o.alloc = self._allocator._alloc
            o.free = self._allocator._free
        self.options = o
        h = C.c_void_p()
        st = lib.cr_create(C.byref(d), C.byref(o), C.byref(h))
        _check(st, None, "cr_create")
        self.h = h
        self.lam = float(lam)

    @classmethod
    def from_problem(cls, p, **kw) -> "ConReg":
        return cls(p.Lx, p.Ly, p.X, p.Y, p.Omega, p.lam, **kw)

    def close(self):
        if getattr(self, "h", None):
            self._lib.cr_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    # ---- Algorithm 1 steps -------------------------------------------------
    def cr_add_rank_one(self) -> dict:
        info = cr_rank1_info()
        st = self._lib.cr_add_rank_one(self.h, C.byref(info))
        if st not in (CR_OK, CR_ENOTCONV):
            _check(st, self.h, "cr_add_rank_one")
        out = {k: getattr(info, k) for k, _ in cr_rank1_info._fields_}
        out["status"] = st
        return out

    def cr_project(self, tol: float) -> dict:
        info = cr_proj_info()
        st = self._lib.cr_project(self.h, float(tol), C.byref(info))
        if st not in (CR_OK, CR_ENOTCONV):
            _check(st, self.h, "cr_project")
        return {"iters": info.iters, "relres": info.relres, "status": st}

    def cr_residual(self, relres=True, J=True, dW=True):
        a, b, c = C.c_double(np.nan), C.c_double(np.nan), C.c_double(np.nan)
        st = self._lib.cr_residual(self.h, C.byref(a) if relres else None, C.byref(b) if J else None,
                                   C.byref(c) if dW else None)
        _check(st, self.h, "cr_residual")
        return {"relres": a.value, "J": b.value, "dW": c.value}

    def cr_solve(self, r_max: int, tau: float, relres_target: float = 0.0) -> dict:
        info = cr_solve_info()
        st = self._lib.cr_solve(self.h, int(r_max), float(tau), float(relres_target), C.byref(info))
        if st not in (CR_OK, CR_ENOTCONV):
            _check(st, self.h, "cr_solve")
        out = {k: getattr(info, k) for k, _ in cr_solve_info._fields_}
        out["stop_name"] = STOP_NAMES.get(info.stop, "?")
        out["status"] = st
        return out

    def cr_get_rank(self) -> int:
        j = C.c_int32()
        _check(self._lib.cr_get_rank(self.h, C.byref(j)), self.h, "cr_get_rank")
        return j.value

    def cr_get_factors(self):
        j = self.cr_get_rank()
        U = np.zeros((self.ny, j), order="F")
        Z = np.zeros((j, j), order="F")
        V = np.zeros((self.nx, j), order="F")
        if j:
            _check(self._lib.cr_get_factors(self.h, _ptr(U), self.ny, _ptr(Z), j, _ptr(V), self.nx), self.h,
                   "cr_get_factors")
        return U, Z, V

    def cr_cv_error(self, Xt, Yt, Omt):
        """(sum_a |(W x_a - y_a) o omega_a|^2, sum_a |y_a o omega_a|^2) over held-out columns."""
        Xt, Yt = _f64(Xt), _f64(Yt)
        Omt = np.asfortranarray(np.asarray(Omt, dtype=np.uint8))
        mt = Xt.shape[1]
        num, den = C.c_double(), C.c_double()
        _check(self._lib.cr_cv_error(self.h, mt, _ptr(Xt), max(1, self.nx), _ptr(Yt), max(1, self.ny),
                                     _ptr(Omt, _up), max(1, self.ny), C.byref(num), C.byref(den)), self.h,
               "cr_cv_error")
        return num.value, den.value

    def cr_svd_factors(self):
        """(U^, sigma, V^): the SVD W = U^ diag(sigma) V^^T of the current solution (Sec. 4)."""
        j = self.cr_get_rank()
        Uh = np.zeros((self.ny, j), order="F")
        Vh = np.zeros((self.nx, j), order="F")
        s = np.zeros(j)
        if j:
            _check(self._lib.cr_svd_factors(self.h, _ptr(Uh), self.ny, _ptr(s), _ptr(Vh), self.nx), self.h,
                   "cr_svd_factors")
        return Uh, s, Vh

    def cr_solution_report(self, nonneg: bool = False, ref=None, want_w: bool = False) -> dict:
        """Statistics of W = U Z V^T (projected onto W >= 0 if ``nonneg``) against the
        reference ``ref`` = (U*, Z*, V*) (None: W* = 0), as a dict with the fields of
        cr_solution_stats; with ``want_w`` also "W_out" = P(W) (ny x nx)."""
        st = cr_solution_stats()
        jr = 0
        Ur = Zr = Vr = None
        if ref is not None:
            Ur, Zr, Vr = (_f64(a) for a in ref)
            jr = Zr.shape[0]
        W = np.zeros((self.ny, self.nx), order="F") if want_w else None
        nul = C.cast(None, _dp)
        _check(self._lib.cr_solution_report(
            self.h, 1 if nonneg else 0, jr,
            _ptr(Ur) if jr else nul, max(1, self.ny), _ptr(Zr) if jr else nul, max(1, jr),
            _ptr(Vr) if jr else nul, max(1, self.nx),
            _ptr(W) if want_w else nul, max(1, self.ny), C.byref(st)), self.h, "cr_solution_report")
        out = {k: getattr(st, k) for k, _ in cr_solution_stats._fields_}
        if want_w:
            out["W_out"] = W
        return out

    @classmethod
    def _adopt(cls, handle, nx: int, ny: int, lam: float) -> "ConReg":
        """Wrap a problem handle that the library created (cr_solve_batch's kept members)."""
        g = cls.__new__(cls)
        g._lib = load()
        g._keep = []
        g._allocator = None
        g.nx, g.ny, g.lam = nx, ny, float(lam)
        g.h = C.c_void_p(handle)
        return g

    def cr_get_state(self) -> bytes:
        """Opaque checkpoint of the iterate (rank, U, Z, V, the previous Z)."""
        n = C.c_size_t(0)
        _check(self._lib.cr_get_state(self.h, None, C.byref(n)), self.h, "cr_get_state")
        buf = C.create_string_buffer(n.value)
        _check(self._lib.cr_get_state(self.h, buf, C.byref(n)), self.h, "cr_get_state")
        return buf.raw[:n.value]

    def cr_set_state(self, state: bytes):
        buf = C.create_string_buffer(bytes(state), len(state))
        _check(self._lib.cr_set_state(self.h, buf, len(state)), self.h, "cr_set_state")

    def cr_set_factors(self, U, Z, V):
        U, Z, V = _f64(U), _f64(Z), _f64(V)
        j = Z.shape[0]
        _check(self._lib.cr_set_factors(self.h, j, _ptr(U), max(1, self.ny), _ptr(Z), max(1, j), _ptr(V),
                                        max(1, self.nx)), self.h, "cr_set_factors")

    def cr_apply_residual(self, vec, trans: bool = False) -> np.ndarray:
        vec = np.ascontiguousarray(vec, dtype=np.float64)
        out = np.zeros(self.nx if trans else self.ny)
        _check(self._lib.cr_apply_residual(self.h, int(trans), _ptr(vec), _ptr(out)), self.h, "cr_apply_residual")
        return out

    def cr_galerkin_assembly(self, method: int = 0) -> np.ndarray:
        """G[a] = U^T diag(Omega_a) U (float32) for the current U; method 0 tensor cores, 1 float64 rounded."""
        j = self.cr_get_rank()
        G = np.zeros((self.m, j, j), dtype=np.float32)
        if j:
            # block a at a*j*j, column-major j x j
            buf = np.zeros(self.m * j * j, dtype=np.float32)
            _check(self._lib.cr_galerkin_assembly(self.h, int(method), buf.ctypes.data_as(C.POINTER(C.c_float)), j),
                   self.h, "cr_galerkin_assembly")
            G = buf.reshape(self.m, j, j).transpose(0, 2, 1).copy()
        return G

    def cr_set_voxel_grid(self, side: int, mask: np.ndarray):
        """Box of the active voxels of `mask` (C order), rows numbered in that order."""
        dims = np.array(list(mask.shape) + [1] * (3 - mask.ndim), dtype=np.int32)
        idx = np.ascontiguousarray(np.flatnonzero(mask.ravel()), dtype=np.int32)
        _check(self._lib.cr_set_voxel_grid(self.h, int(side), _ptr(dims, _ip), _ptr(idx, _ip)), self.h,
               "cr_set_voxel_grid")

    def cr_set_preconditioner(self, net):
        _check(self._lib.cr_set_preconditioner(self.h, net.h if net is not None else None), self.h,
               "cr_set_preconditioner")
        self._net = net

    def cr_get_stats(self, reset: bool = False) -> dict:
        s = cr_stats()
        _check(self._lib.cr_get_stats(self.h, C.byref(s), int(reset)), self.h, "cr_get_stats")
        return {"launches": s.launches, "pcg_solves": s.pcg_solves, "pcg_iters": s.pcg_iters,
                "h2d_bytes": s.h2d_bytes, "d2h_bytes": s.d2h_bytes,
                "phase_ms": {PHASES[i]: s.phase_ms[i] for i in range(len(PHASES))},
                "phase_calls": {PHASES[i]: s.phase_calls[i] for i in range(len(PHASES))},
                "learned_solves": s.learned_solves, "learned_fallbacks": s.learned_fallbacks,
                "learned_off": s.learned_off, "mixed_handovers": s.mixed_handovers,
                "pcg_cluster": [s.pcg_cluster[0], s.pcg_cluster[1]],
                "pcg_multigrid": [s.pcg_multigrid[0], s.pcg_multigrid[1]],
                "galerkin_eigen": [s.galerkin_eigen[0], s.galerkin_eigen[1]],
                "pcg_iters_side": [s.pcg_iters_side[0], s.pcg_iters_side[1]],
                "pcg_bytes_per_iter": [s.pcg_bytes_per_iter[0], s.pcg_bytes_per_iter[1]]}

    def cr_solve_u(self, v, rhs, allow_notconv: bool = False):
        """(solution, iterations); with ``allow_notconv`` a solve that stopped at
        pcg_maxit returns (best iterate, iterations, status) instead of raising."""
        v = np.ascontiguousarray(v, dtype=np.float64)
        rhs = np.ascontiguousarray(rhs, dtype=np.float64)
        out = np.zeros(self.ny)
        it = C.c_int32()
        st = self._lib.cr_solve_u(self.h, _ptr(v), _ptr(rhs), _ptr(out), C.byref(it))
        if allow_notconv and st == CR_ENOTCONV:
            return out, it.value, st
        _check(st, self.h, "cr_solve_u")
        return (out, it.value, st) if allow_notconv else (out, it.value)

    def cr_solve_v(self, u, rhs, allow_notconv: bool = False):
        """(solution, iterations); with ``allow_notconv`` a solve that stopped at
        pcg_maxit returns (best iterate, iterations, status) instead of raising."""
        u = np.ascontiguousarray(u, dtype=np.float64)
        rhs = np.ascontiguousarray(rhs, dtype=np.float64)
        out = np.zeros(self.nx)
        it = C.c_int32()
        st = self._lib.cr_solve_v(self.h, _ptr(u), _ptr(rhs), _ptr(out), C.byref(it))
        if allow_notconv and st == CR_ENOTCONV:
            return out, it.value, st
        _check(st, self.h, "cr_solve_v")
        return (out, it.value, st) if allow_notconv else (out, it.value)


def solve_batch(p, members, r_max: int, tau: float = 0.0, relres_target: float = 0.0, concurrency: int = 0,
                keep: bool = False, stream=None, **opts):
    """cr_solve_batch on the data set of problem ``p`` (Lx, Ly, X, Y, Omega).

    ``members``: list of (lambda, fit_cols, test_cols).  Returns one dict per
    member (status, rank, stop, relres, dW, J, cv_num, cv_den, cv, pcg_iters,
    cg_iters, seconds, slot); with ``keep`` also a list of ConReg handles on the
    members' solved problems (the caller closes them).  Device memory comes from
    the library's own allocator (the workers run outside Python)."""
    import torch

    if not torch.cuda.is_available():
        raise RuntimeError("solve_batch needs a CUDA device")
    lib = load()
    X = _f64(p.X)
    Y = _f64(p.Y)
    Om = np.asfortranarray(np.asarray(p.Omega, dtype=np.uint8))
    hold = [X, Y, Om]
    d = cr_problem_desc()
    d.nx, d.ny, d.ninj = X.shape[0], Y.shape[0], X.shape[1]
    for name, L in (("Lx", p.Lx), ("Ly", p.Ly)):
        rp = np.ascontiguousarray(L.rowptr, dtype=np.int32)
        co = np.ascontiguousarray(L.col, dtype=np.int32)
        va = np.ascontiguousarray(L.val, dtype=np.float64)
        hold += [rp, co, va]
        setattr(d, name, cr_csr(L.n, _ptr(rp, _ip), _ptr(co, _ip), _ptr(va)))
    d.X_host, d.ldx = _ptr(X), d.nx
    d.Y_host, d.ldy = _ptr(Y), d.ny
    d.Omega_host, d.ldo = _ptr(Om, _up), d.ny
    d.lambda_ = 1.0
    if stream is None:
        stream = torch.cuda.current_stream()
    o = default_options(**opts)
    o.stream = C.c_void_p(stream.cuda_stream)
    n = len(members)
    arr = (cr_member * max(n, 1))()
    for k, (lam, fit, test) in enumerate(members):
        fa = np.ascontiguousarray(fit, dtype=np.int32)
        ta = np.ascontiguousarray(test if test is not None else [], dtype=np.int32)
        hold += [fa, ta]
        arr[k] = cr_member(float(lam), _ptr(fa, _ip), len(fa), _ptr(ta, _ip) if len(ta) else None, len(ta))
    res = (cr_member_result * max(n, 1))()
    handles = (C.c_void_p * max(n, 1))() if keep else None
    st = lib.cr_solve_batch(C.byref(d), C.byref(o), arr, n, int(r_max), float(tau), float(relres_target),
                            int(concurrency), res, handles)
    out = []
    for k in range(n):
        r = res[k]
        out.append({"status": r.status, "rank": r.rank, "stop": r.stop, "stop_name": STOP_NAMES.get(r.stop, "?"),
                    "relres": r.relres, "dW": r.dW, "J": r.J, "cv_num": r.cv_num, "cv_den": r.cv_den,
                    "cv": r.cv_num / r.cv_den if r.cv_den > 0 else float("nan"), "pcg_iters": r.pcg_iters,
                    "cg_iters": r.cg_iters, "seconds": r.seconds, "slot": r.slot})
    kept = []
    if keep:
        kept = [ConReg._adopt(handles[k], d.nx, d.ny, members[k][0]) if handles[k] else None for k in range(n)]
    if st not in (CR_OK, CR_ENOTCONV):
        for g in kept:
            if g is not None:
                g.close()
        _check(st, None, "cr_solve_batch")
    return (out, kept) if keep else out


def cr_lambda_from_bar(lam_bar: float, ninj: int, nx: int) -> float:
    return load().cr_lambda_from_bar(float(lam_bar), int(ninj), int(nx))


def arrow_check(d, z, alpha):
    """The device arrowhead eigen-decomposition (cr_arrow_check): (mu, W)."""
    lib = load()
    d = np.ascontiguousarray(d, dtype=np.float64)
    z = np.ascontiguousarray(z, dtype=np.float64)
    n = d.size
    mu = np.zeros(n + 1)
    W = np.zeros((n + 1, n + 1), order="F")
    _check(lib.cr_arrow_check(n, _ptr(d), _ptr(z), float(alpha), _ptr(mu), W.ctypes.data_as(_dp)), None,
           "cr_arrow_check")
    return mu, W


class ConvNet:
    """The learned preconditioner's network (cr_net_*): 2 -> 16 -> 16 -> 16 -> 1
    channels of 3x3x3 convolutions on a D x H x W box, trained on the GPU."""

    def __init__(self, dims, batch_cap: int = 8, seed: int = 1808, stream=None):
        import torch

        self._lib = load()
        d = list(dims) + [1] * (3 - len(dims))
        self.dims = tuple(int(x) for x in d)
        if stream is None:
            stream = torch.cuda.current_stream()
        self.stream = stream
        h = C.c_void_p()
        _check(self._lib.cr_net_create(self.dims[0], self.dims[1], self.dims[2], int(batch_cap), int(seed),
                                       C.c_void_p(stream.cuda_stream), C.byref(h)), None, "cr_net_create")
        self.h = h
        self.V = self.dims[0] * self.dims[1] * self.dims[2]

    def close(self):
        if getattr(self, "h", None):
            self._lib.cr_net_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @staticmethod
    def param_count() -> int:
        return load().cr_net_param_count()

    def get_params(self) -> np.ndarray:
        out = np.zeros(self.param_count(), dtype=np.float32)
        _check(self._lib.cr_net_get_params(self.h, out.ctypes.data_as(C.POINTER(C.c_float)), out.size), None,
               "cr_net_get_params")
        return out

    def set_params(self, w: np.ndarray):
        w = np.ascontiguousarray(w, dtype=np.float32)
        _check(self._lib.cr_net_set_params(self.h, w.ctypes.data_as(C.POINTER(C.c_float)), w.size), None,
               "cr_net_set_params")

    def forward(self, x):
        """x: torch float32 (B, 2, D, H, W) on the GPU -> (B, D, H, W)."""
        import torch

        x = x.contiguous()
        out = torch.empty((x.shape[0],) + self.dims, dtype=torch.float32, device=x.device)
        _check(self._lib.cr_net_forward(self.h, x.shape[0], x.data_ptr(), out.data_ptr()), None, "cr_net_forward")
        return out

    def gradients(self, x, target, mask):
        """Loss and parameter gradients (numpy, cr_net_param_count entries)."""
        g = np.zeros(self.param_count(), dtype=np.float32)
        loss = C.c_float()
        _check(self._lib.cr_net_gradients(self.h, x.shape[0], x.contiguous().data_ptr(), target.contiguous().data_ptr(),
                                          mask.contiguous().data_ptr(), C.byref(loss),
                                          g.ctypes.data_as(C.POINTER(C.c_float))), None, "cr_net_gradients")
        return loss.value, g

    @staticmethod
    def check_f64(dims, params, x, target, mask):
        """The same kernel templates in float64 (cr_net_check_f64), host arrays in and
        out: params (float64, packed as get_params), x (B, 2, D, H, W), target
        (B, D, H, W), mask (D, H, W) -> (out (B, D, H, W), loss, gradients)."""
        lib = load()
        d = list(dims) + [1] * (3 - len(dims))
        x = np.ascontiguousarray(x, dtype=np.float64)
        t = np.ascontiguousarray(target, dtype=np.float64)
        m = np.ascontiguousarray(mask, dtype=np.uint8)
        p = np.ascontiguousarray(params, dtype=np.float64)
        B = x.shape[0]
        out = np.zeros((B,) + tuple(d), dtype=np.float64)
        grads = np.zeros(p.size, dtype=np.float64)
        loss = C.c_double()
        _check(lib.cr_net_check_f64(d[0], d[1], d[2], B, _ptr(p), _ptr(x), _ptr(t), _ptr(m, _up), _ptr(out),
                                    C.byref(loss), _ptr(grads)), None, "cr_net_check_f64")
        return out, loss.value, grads

    def train_step(self, x, target, mask, lr: float) -> float:
        loss = C.c_float()
        _check(self._lib.cr_net_train_step(self.h, x.shape[0], x.contiguous().data_ptr(), target.contiguous().data_ptr(),
                                           mask.contiguous().data_ptr(), float(lr), C.byref(loss)), None,
               "cr_net_train_step")
        return loss.value
