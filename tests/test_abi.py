"""CPU-side checks of the C ABI: the library loads, exports every function that
include/conreg.h declares, and rejects invalid problems before touching a GPU."""
import ctypes as C
import os
import re

import numpy as np
import pytest

from paper_1808_05510_gb300 import build as B
from paper_1808_05510_gb300 import conreg as cr
from paper_1808_05510_gb300 import synth

HDR = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "conreg.h")


@pytest.fixture(scope="module")
def lib():
    B.build()
    return cr.load()


def declared_functions():
    txt = open(HDR).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(cr_[a-z_0-9]+)\s*\(", txt)))


def test_header_matches_binding_and_exports(lib):
    decl = declared_functions()
    assert decl, "no declarations parsed"
    assert set(decl) == set(cr.SIGNATURES), set(decl) ^ set(cr.SIGNATURES)
    for name in decl:
        assert hasattr(lib, name), name


def test_options_and_helpers(lib):
    o = cr.default_options()
    assert o.struct_size == C.sizeof(cr.cr_options)
    assert o.als_delta == 0.1 and o.als_max_iter == 10 and o.pcg_tol == 1e-10
    assert lib.cr_lambda_from_bar(1e6, 126, 22377) == pytest.approx(1e6 * 126 / 22377)
    assert lib.cr_status_str(cr.CR_EINVAL) == b"invalid argument"


def _desc(p, **over):
    keep = []
    d = cr.cr_problem_desc()
    d.nx, d.ny, d.ninj = p.nx, p.ny, p.m
    for name, L in (("Lx", p.Lx), ("Ly", p.Ly)):
        rp = np.ascontiguousarray(over.get(name + "_rowptr", L.rowptr), dtype=np.int32)
        co = np.ascontiguousarray(over.get(name + "_col", L.col), dtype=np.int32)
        va = np.ascontiguousarray(over.get(name + "_val", L.val), dtype=np.float64)
        keep += [rp, co, va]
        setattr(d, name, cr.cr_csr(L.n, cr._ptr(rp, cr._ip), cr._ptr(co, cr._ip), cr._ptr(va)))
    X = np.asfortranarray(over.get("X", p.X), dtype=np.float64)
    Y = np.asfortranarray(over.get("Y", p.Y), dtype=np.float64)
    Om = np.asfortranarray(over.get("Omega", p.Omega), dtype=np.uint8)
    keep += [X, Y, Om]
    d.X_host, d.ldx = cr._ptr(X), p.nx
    d.Y_host, d.ldy = cr._ptr(Y), p.ny
    d.Omega_host, d.ldo = cr._ptr(Om, cr._up), p.ny
    d.lambda_ = over.get("lam", p.lam)
    return d, keep


@pytest.mark.parametrize("case", ["nan_x", "inf_y", "omega2", "lam0", "lamneg", "nonsym", "badcol", "rcap",
                                  "mem_kind", "grid_dup", "grid_box", "galerkin_form"])
def test_create_rejects_invalid_input(lib, case):
    p = synth.rect2d()
    over = {}
    opts = cr.default_options(r_cap=4)
    if case == "nan_x":
        X = p.X.copy(); X[3, 1] = np.nan; over["X"] = X
    elif case == "inf_y":
        Y = p.Y.copy(); Y[0, 0] = np.inf; over["Y"] = Y
    elif case == "omega2":
        Om = p.Omega.copy(); Om[2, 2] = 2; over["Omega"] = Om
    elif case == "lam0":
        over["lam"] = 0.0
    elif case == "lamneg":
        over["lam"] = -1.0
    elif case == "nonsym":
        val = p.Lx.val.copy(); val[1] = -2.0; over["Lx_val"] = val
    elif case == "badcol":
        col = p.Ly.col.copy(); col[0] = p.ny + 5; over["Ly_col"] = col
    elif case == "rcap":
        opts = cr.default_options(r_cap=p.nx + 1)
    elif case == "galerkin_form":
        opts = cr.default_options(r_cap=4, galerkin_form=3)
    d, keep = _desc(p, **over)
    if case == "mem_kind":
        d.mem_kind = 7
    elif case in ("grid_dup", "grid_box"):
        idx = np.arange(p.ny, dtype=np.int32)
        if case == "grid_dup":
            idx[1] = idx[0]  # two rows on one voxel
        keep.append(idx)
        d.grid_y.dims[:] = (1, 9, 7) if case == "grid_dup" else (1, 2, 2)  # grid_box: box smaller than the rows
        d.grid_y.box_index = cr._ptr(idx, cr._ip)
    h = C.c_void_p()
    st = lib.cr_create(C.byref(d), C.byref(opts), C.byref(h))
    assert st == cr.CR_EINVAL
    assert not h.value
    assert lib.cr_last_error(None)


def test_destroy_null_is_noop(lib):
    lib.cr_destroy(None)


STRUCTS = ["cr_csr", "cr_grid", "cr_problem_desc", "cr_options", "cr_rank1_info", "cr_proj_info", "cr_stats", "cr_solve_info",
           "cr_member", "cr_member_result", "cr_solution_stats"]


def test_struct_layouts_match_header(tmp_path):
    """Every ctypes structure of the binding has the size and field offsets
    that a C compiler gives the header's struct (binding drift would silently
    garble the fields after the first mismatch)."""
    import shutil
    import subprocess

    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    lines = ['#include <stddef.h>', '#include <stdio.h>', '#include "conreg.h"', "int main(void) {"]
    for name in STRUCTS:
        lines.append(f'  printf("{name} %zu\\n", sizeof({name}));')
        for field, _ in getattr(cr, name)._fields_:
            cfield = field.rstrip("_")
            lines.append(f'  printf("{name}.{field} %zu\\n", offsetof({name}, {cfield}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-std=c99", "-I", os.path.dirname(HDR), str(src), "-o", str(exe)], check=True)
    out = dict(line.split() for line in subprocess.run([str(exe)], capture_output=True, text=True,
                                                       check=True).stdout.splitlines())
    for name in STRUCTS:
        st = getattr(cr, name)
        assert int(out[name]) == C.sizeof(st), name
        for field, _ in st._fields_:
            assert int(out[f"{name}.{field}"]) == getattr(st, field).offset, f"{name}.{field}"
