"""Representative kernel cases for profiling runs (ncu) on the visual-cortex workload.

    python -m paper_1808_05510_gb300.profile_cases pcg fp64|mixed [jacobi|auto]
        one u-side and one v-side ALS solve (Eqs. ALS_linsys, ALS_linsys_v) for the
        first ALS vector v = R_0^T 1 / |R_0^T 1|, to relative residual 1e-8, twice;
        jacobi (default): Jacobi PCG on both sides; auto: the automatic choice
        (multigrid PCG on the v side, pcg_mg_kernel); prints iterations and the
        CUDA-event time of each solve
    python -m paper_1808_05510_gb300.profile_cases galerkin fp64|mixed [eigen|jacobi]
        two Galerkin projections (Eq. Proj_Sylv) at rank 60 from a float64 greedy run,
        in the eigenbasis form (default) or the original-basis Jacobi form
    python -m paper_1808_05510_gb300.profile_cases galerkin_scan fp64|mixed
        one projection at each of j = 60, 100, 250, 500 in both forms (CUDA-event
        phase times): iterations and time per CG iteration
    python -m paper_1808_05510_gb300.profile_cases assembly tc
        three tensor-core assemblies of G_a = U^T diag(Omega_a) U at rank 100
    python -m paper_1808_05510_gb300.profile_cases post fp64
        three solution passes (W = U Z V^T in float64 tiles, projected onto W >= 0,
        statistics only) at rank 100 with random orthonormal U, V; prints the
        CUDA-event time of each call
    python -m paper_1808_05510_gb300.profile_cases pcg_stress fp32|fp64 [solves]
        u-side ALS solves on the ~4M-voxel stress shell (grid-wide PCG, vectors in
        HBM): fp32 = one float32 grid solve to 1e-5 inside the mixed form's
        refinement, fp64 = float64 grid solve to 1e-5; prints iterations and the
        CUDA-event time of each solve
"""
from __future__ import annotations

import sys

import numpy as np


def pcg(form: str, precond: str = "jacobi") -> None:
    import torch

    from . import synth
    from .conreg import CR_FP64, CR_MIXED, CR_PRECOND_AUTO, CR_PRECOND_JACOBI, ConReg

    p = synth.visual_cortex()
    prec = CR_MIXED if form == "mixed" else CR_FP64
    pc = CR_PRECOND_AUTO if precond == "auto" else CR_PRECOND_JACOBI
    with ConReg.from_problem(p, r_cap=4) as g0:
        v = g0.cr_apply_residual(np.ones(p.ny), trans=True)
        v /= np.linalg.norm(v)
        rhs_u = g0.cr_apply_residual(v)
        u = rhs_u / np.linalg.norm(rhs_u)
        rhs_v = g0.cr_apply_residual(u, trans=True)
    with ConReg.from_problem(p, r_cap=4, precision=prec, pcg_tol=1e-8, precond=pc) as g:
        stream = g.stream
        for _ in range(2):
            out = []
            for solve, a, b in ((g.cr_solve_u, v, rhs_u), (g.cr_solve_v, u, rhs_v)):
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                _, it = solve(a, b)
                e1.record(stream)
                e1.synchronize()
                out.append((it, round(e0.elapsed_time(e1), 3)))
            print("iterations, ms (u, v):", out, "multigrid levels:", g.cr_get_stats()["pcg_multigrid"], flush=True)


def galerkin(form: str, gform: str = "eigen") -> None:
    from . import synth
    from .conreg import CR_FP64, CR_GALERKIN_EIGEN, CR_GALERKIN_JACOBI, CR_MIXED, ConReg

    p = synth.visual_cortex()
    with ConReg.from_problem(p, r_cap=100) as g:
        g.cr_solve(60, 1e-9, 0.0)
        U, Z, V = g.cr_get_factors()
    prec = CR_MIXED if form == "mixed" else CR_FP64
    gf = CR_GALERKIN_JACOBI if gform == "jacobi" else CR_GALERKIN_EIGEN
    with ConReg.from_problem(p, r_cap=100, precision=prec, galerkin_form=gf) as g:
        for k in range(2):
            g.cr_set_factors(U, Z * (1.0 + 1e-3 * (k + 1)), V)
            print(g.cr_project(5e-10), flush=True)


def galerkin_scan(form: str) -> None:
    """Galerkin projections at j = 60, 100, 250, 500 on the visual-cortex workload
    from orthonormal smoothed-noise factors and a small Z, to relative residual
    5e-10, in both forms: CG iterations, the Galerkin phase's device time (CUDA
    events, profile mode) without the eigenbasis build, and the time per iteration."""
    import json

    import scipy.sparse as sp

    from . import synth
    from .conreg import CR_FP64, CR_GALERKIN_EIGEN, CR_GALERKIN_JACOBI, CR_MIXED, ConReg

    p = synth.visual_cortex()
    rng = np.random.default_rng(7)

    def basis(L, j):
        A = sp.csr_matrix((L.val, L.col, L.rowptr), shape=(L.n, L.n))
        W = rng.standard_normal((L.n, j))
        d = A.diagonal().max()
        for _ in range(3):
            W = W - (A @ W) / (2 * d)
        return np.linalg.qr(W)[0]

    prec = CR_MIXED if form == "mixed" else CR_FP64
    for j in (60, 100, 250, 500):
        U, V = basis(p.Ly, j), basis(p.Lx, j)
        Z = 1e-3 * rng.standard_normal((j, j))
        for name, gf in (("eigen", CR_GALERKIN_EIGEN), ("jacobi", CR_GALERKIN_JACOBI)):
            with ConReg.from_problem(p, r_cap=j, precision=prec, galerkin_form=gf, profile=1) as g:
                g.cr_set_factors(U, Z, V)
                g.cr_get_stats(reset=True)
                info = g.cr_project(5e-10)
                st = g.cr_get_stats()
            ms = st["phase_ms"]["galerkin"] - st["phase_ms"]["basis"]
            print(json.dumps({"j": j, "form": name, "precision": form, "iters": info["iters"],
                              "galerkin_ms": round(ms, 3), "basis_ms": round(st["phase_ms"]["basis"], 3),
                              "us_per_iter": round(1e3 * ms / max(info["iters"], 1), 2)}), flush=True)


def assembly(form: str) -> None:
    """Tensor-core Galerkin assembly at rank 100 (random orthonormal U), three times."""
    from . import synth
    from .conreg import CR_MIXED, ConReg

    p = synth.visual_cortex()
    j = 100
    rng = np.random.default_rng(7)
    U, _ = np.linalg.qr(rng.standard_normal((p.ny, j)))
    V, _ = np.linalg.qr(rng.standard_normal((p.nx, j)))
    with ConReg.from_problem(p, r_cap=j, precision=CR_MIXED) as g:
        g.cr_set_factors(U, np.eye(j), V)
        for _ in range(3):
            G = g.cr_galerkin_assembly(0 if form != "fp64" else 1)
        print("assembled", G.shape, flush=True)


def post(form: str) -> None:
    import torch

    from . import synth
    from .conreg import ConReg

    p = synth.visual_cortex()
    j = 100
    rng = np.random.default_rng(11)
    U, _ = np.linalg.qr(rng.standard_normal((p.ny, j)))
    V, _ = np.linalg.qr(rng.standard_normal((p.nx, j)))
    Z = rng.standard_normal((j, j))
    with ConReg.from_problem(p, r_cap=j) as g:
        g.cr_set_factors(U, Z, V)
        for _ in range(3):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record(g.stream)
            r = g.cr_solution_report(nonneg=True)
            e1.record(g.stream)
            e1.synchronize()
            print(f"entries {r['entries']} negative {r['n_negative']} call_ms {e0.elapsed_time(e1):.3f}", flush=True)


def pcg_stress(form: str, solves: int = 2) -> None:
    import torch

    from . import synth
    from .conreg import CR_FP64, CR_MIXED, ConReg

    p = synth.stress_shell()
    v = p.X.sum(axis=1)
    v /= np.linalg.norm(v)
    rhs = np.random.default_rng(3).standard_normal(p.ny)
    prec = CR_MIXED if form == "fp32" else CR_FP64
    # mixed: outer tolerance at the inner one, so each solve is one float32 grid launch
    with ConReg.from_problem(p, r_cap=2, precision=prec, pcg_tol=1e-5, pcg_maxit=200000, profile=1) as g:
        for _ in range(solves):
            g.cr_get_stats(reset=True)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(g.stream)
            _, it = g.cr_solve_u(v, rhs)
            e1.record(g.stream)
            e1.synchronize()
            st = g.cr_get_stats()
            kms, kn = st["phase_ms"]["pcg_kernel"], st["phase_calls"]["pcg_kernel"]
            print(f"voxels {p.ny} iterations {it} solve_ms {e0.elapsed_time(e1):.3f} "
                  f"pcg_phase_ms {st['phase_ms']['pcg_u']:.3f} kernel_ms {kms:.3f} launches {kn} "
                  f"kernel_us_per_iter {1e3 * kms / max(it, 1):.1f}", flush=True)


if __name__ == "__main__":
    case, form = sys.argv[1], (sys.argv[2] if len(sys.argv) > 2 else "fp64")
    if case == "pcg_stress":
        pcg_stress(form, int(sys.argv[3]) if len(sys.argv) > 3 else 2)
    else:
        extra = sys.argv[3:4]
        {"pcg": pcg, "galerkin": galerkin, "galerkin_scan": galerkin_scan, "assembly": assembly,
         "post": post}[case](form, *extra)
