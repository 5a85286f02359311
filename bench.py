#!/usr/bin/env python
"""Benchmark of the greedy low-rank connectome-regression solver on GB300.

One step = one complete run of Algorithm 1 (ALS rank-one updates with PCG
sub-solves, orthogonalisation, Galerkin projection, residual and stopping test)
from W = 0 up to relres <= target, dW <= tau or r_max, on the visual-cortex-
shaped synthetic workload (~7,500 voxels in a smooth random blob mask of a 40^3
box, 7-point Laplacians, 28 Gaussian injections, lambda = 100, rank <= 100).

Reported: rank-1 updates per second (whole job, all GPUs), the time to the
relative residual target when reached, an end-to-end number through the public
API with host buffers, the roofline of the dominant kernel (the PCG kernel of
the side with the larger share of the step),
the CPU float64 oracle as a baseline, SM clocks during the timed region, and
the number of library kernel launches.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

For N > 1 (torchrun, one process per GPU) every rank solves its own replica
of the workload (a single greedy solve is a chain of dependent steps with a
global reduction in every PCG iteration, so it does not shard) and rank 0
reports the aggregate over ranks divided by the slowest rank's time.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_1808_05510_gb300 import replicas  # noqa: E402  (host-side cross-rank scalars only)

METRIC = "time-to-rel-residual 1e-6 and rank-1 updates/s, mixed/learned vs plain FP64 GPU"
UNIT = "rank-1 updates/s"


def parse(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--lam", type=float, default=1e2)
    ap.add_argument("--r-max", type=int, default=100)
    ap.add_argument("--tau", type=float, default=1e-9)
    ap.add_argument("--relres", type=float, default=1e-6)
    ap.add_argument("--precision", default="mixed", choices=["fp64", "mixed"],
                    help="form reported as the headline value; the float64 form is always measured beside it")
    ap.add_argument("--cpu-seconds", type=float, default=20.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-learned", action="store_true")
    ap.add_argument("--no-batch", action="store_true")
    ap.add_argument("--no-ttr", action="store_true")
    ap.add_argument("--no-post", action="store_true", help="skip the post-processing measurement")
    ap.add_argument("--batch-r", type=int, default=50, help="rank of every sweep member in the batched form")
    ap.add_argument("--learn-steps", type=int, default=200)
    ap.add_argument("--precond", default="auto", choices=["auto", "multigrid", "jacobi"],
                    help="preconditioner of the ALS sub-solves in the headline forms")
    ap.add_argument("--no-jacobi", action="store_true", help="skip the Jacobi-PCG forms timed beside the headline")
    ap.add_argument("--resid-every", type=int, default=0,
                    help="timed forms and end-to-end leg: evaluate relres every k greedy steps, 0 = the library's "
                         "automatic schedule (dW every step; relres always at the rank cap)")
    ap.add_argument("--ttr-r", type=int, default=500, help="rank cap of the visual-cortex time to relres 1e-6")
    ap.add_argument("--ttr-resid-every", type=int, default=0,
                    help="visual-cortex time to relres: evaluate relres every k greedy steps, 0 = the library's "
                         "automatic schedule (dW every step)")
    ap.add_argument("--no-cortex", action="store_true", help="skip the whole-cortex line")
    ap.add_argument("--cortex-r", type=int, default=300, help="rank cap of the whole-cortex line")
    ap.add_argument("--cortex-resid-every", type=int, default=0,
                    help="whole-cortex: evaluate relres every k greedy steps, 0 = automatic (dW every step)")
    return ap.parse_args(argv)


def parse_args_list(argv):
    return parse(argv)


def workload(args, rank=0):
    from paper_1808_05510_gb300 import synth

    p = synth.visual_cortex(seed=1810 + rank, lam=args.lam, r_max=args.r_max)
    cfg = {
        "workload": "visual-cortex-shaped synthetic: smooth random blob mask in a 40^3 box, 7-point Laplacians",
        "ny": p.ny, "nx": p.nx, "ninj": p.m, "lambda": p.lam, "r_max": args.r_max, "tau": args.tau,
        "relres_target": args.relres, "precision": args.precision, "pcg_tol": 1e-10, "pcg_tol_mixed": "1e-10 (float32 inner solves to max(1e-5, what the float64 target still needs / 2) under float64 refinement)",
        "l2": "flushed between steps (256 MiB write)", "parallelism": "replicas",
    }
    return p, cfg


# ----------------------------------------------------------------------------- helpers
class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.samples = []
        self._stop = threading.Event()
        self._t = threading.Thread(target=self._run, daemon=True)

    def _run(self):
        while not self._stop.is_set():
            try:
                out = subprocess.run(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                      "--format=csv,noheader,nounits"], capture_output=True, text=True,
                                     timeout=5).stdout.strip()
                if out:
                    self.samples.append([x.strip() for x in out.split(",")])
            except Exception:
                pass
            self._stop.wait(0.2)

    def __enter__(self):
        self._t.start()
        return self

    def __exit__(self, *a):
        self._stop.set()
        self._t.join(timeout=10)

    def summary(self):
        if not self.samples:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        sm = [float(s[1]) for s in self.samples if s[1].replace(".", "").isdigit()]
        mx = [float(s[2]) for s in self.samples if s[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for s in self.samples for k in range(4) if len(s) > 5 + k and "Active" in s[5 + k]
                          and "Not" not in s[5 + k]})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.samples)}


def flush_l2(buf):
    buf.add_(1.0)


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "of measured"
    except Exception:
        return 6800.0, "of fallback"


KERNEL_SOURCES = {"pcg_reg_kernel": "cr_pcg.cu", "pcg_mg_kernel": "cr_mg.cu", "pcg_grid_kernel": "cr_pcg_grid.cu"}


def pcg_traffic(kernel: str, form: str, side: int):
    """DRAM bytes per launch of `kernel` from the committed ncu summary
    (profiles/<kernel>_traffic.json), or None when there is none or the kernel's
    source has changed since the counters were taken."""
    import hashlib

    try:
        with open(os.path.join(ROOT, "profiles", kernel + "_traffic.json")) as f:
            d = json.load(f)
        src = KERNEL_SOURCES[kernel]
        with open(os.path.join(ROOT, "paper_1808_05510_gb300", "csrc", src), "rb") as f:
            h = hashlib.sha256(f.read()).hexdigest()[:16]
        if h != d["source_sha256_16"]:
            return None
        b = d["dram_bytes_per_launch"]
        key = ("fp64" if form == "fp64" else "f32") + ("_u" if side == 0 else "_v")
        return b.get(key)
    except Exception:
        return None


# ----------------------------------------------------------------------------- CPU oracle
def oracle_sample(p, args, seconds: float, max_steps: int = 0):
    """The CPU float64 oracle (Algorithm 1, its own CG sub-solves) on a bounded
    sample: greedy steps from W = 0 until `seconds` of work (or max_steps steps);
    rank-1 updates/s."""
    from oracle import Oracle

    class Stop(Exception):
        pass

    o = Oracle.from_problem(p, cg_tol=1e-10)
    t0 = time.perf_counter()
    done = [0]

    def cb(st, U, Z, V):
        done[0] = st.j
        if (max_steps and st.j >= max_steps) or (not max_steps and time.perf_counter() - t0 > seconds):
            raise Stop()

    try:
        o.greedy(r_max=args.r_max, tau=args.tau, relres_target=args.relres, callback=cb)
    except Stop:
        pass
    el = time.perf_counter() - t0
    cores = os.cpu_count()
    return {"value": done[0] / el if el > 0 else None, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"first {done[0]} greedy steps of the same workload ({el:.1f} s, numpy/scipy float64, "
                      f"dense residual each step, CG sub-solves to 1e-10)", "steps": done[0], "seconds": el}


# ----------------------------------------------------------------------------- main arms
def run_reference(args, rank, world):
    if rank != 0:
        return
    p, cfg = workload(args)
    for _ in range(max(0, args.warmup)):
        pass  # the oracle has no warm-up state; each sample starts from W = 0
    vals, times = [], []
    per = max(5.0, args.cpu_seconds / max(1, args.steps))
    tot_steps, tot_s = 0, 0.0
    for _ in range(args.steps):
        r = oracle_sample(p, args, per)
        tot_steps += r["steps"]
        tot_s += r["seconds"]
    v = tot_steps / tot_s if tot_s > 0 else None
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot_s / max(1, args.steps),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": cfg,
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
                             "sample": f"{tot_steps} greedy steps in {args.steps} samples of ~{per:.0f} s"},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_ours(args, rank, world, local_rank):
    import numpy as np
    import torch

    from paper_1808_05510_gb300 import build
    from paper_1808_05510_gb300.conreg import ConReg

    build.build()
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    p, cfg = workload(args, rank)
    stream = torch.cuda.current_stream()
    l2buf = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    from paper_1808_05510_gb300.conreg import (CR_FP64, CR_MIXED, CR_PRECOND_AUTO, CR_PRECOND_JACOBI,
                                               CR_PRECOND_LEARNED, CR_PRECOND_MULTIGRID)

    head_pc = {"auto": CR_PRECOND_AUTO, "multigrid": CR_PRECOND_MULTIGRID, "jacobi": CR_PRECOND_JACOBI}[args.precond]

    def measure(prec, net=None, steps=None, warmup=None, precond=None):
        steps = args.steps if steps is None else steps
        warmup = args.warmup if warmup is None else warmup
        pc = CR_PRECOND_LEARNED if net is not None else (head_pc if precond is None else precond)
        g = ConReg.from_problem(p, r_cap=args.r_max, profile=1, precision=prec, precond=pc,
                                residual_every=args.resid_every)
        if net is not None:
            g.cr_set_voxel_grid(0, p.grid_y.mask)
            g.cr_set_voxel_grid(1, p.grid_x.mask)
            g.cr_set_preconditioner(net)

        def one_step():
            g.cr_set_factors(np.zeros((p.ny, 0)), np.zeros((0, 0)), np.zeros((p.nx, 0)))
            return g.cr_solve(args.r_max, args.tau, args.relres)

        for _ in range(warmup):
            one_step()
            flush_l2(l2buf)
        torch.cuda.synchronize()
        g.cr_get_stats(reset=True)
        if world > 1:
            import torch.distributed as dist
            dist.barrier()
        torch.cuda.synchronize()
        ms, infos = [], []
        with ClockSampler(local_rank) as clk:
            for _ in range(steps):
                flush_l2(l2buf)
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                info = one_step()
                e1.record(stream)
                e1.synchronize()
                ms.append(e0.elapsed_time(e1))
                infos.append(info)
        torch.cuda.synchronize()
        stats = g.cr_get_stats(reset=True)
        g.close()
        tot_ms = sum(ms)
        ranks = sum(i["rank"] for i in infos)
        if world > 1:
            import torch.distributed as dist
            dist.barrier()
        all_ranks, t_max = replicas.aggregate(ranks, tot_ms, world, dev)
        value = all_ranks / (t_max / 1e3)
        reached = [i for i in infos if i["stop_name"] == "relres"]
        ttr = (sum(m for m, i in zip(ms, infos) if i["stop_name"] == "relres") / len(reached) / 1e3) if reached else None
        # each side's PCG kernel launches (CUDA events around each launch, on the
        # problem's stream); the mixed form's sub-solves are several float32
        # launches inside float64 refinement.  Algorithmic bytes per iteration come
        # from the library (the multigrid hierarchy's sizes, or the Jacobi count).
        pcg_ms = stats["phase_ms"]["pcg_u"] + stats["phase_ms"]["pcg_v"]
        kern_ms = stats["phase_ms"]["pcg_kernel"] + stats["phase_ms"]["pcg_kernel_v"]
        sides = []
        for side, ph in ((0, "pcg_kernel"), (1, "pcg_kernel_v")):
            kms = stats["phase_ms"][ph]
            calls = max(1, stats["phase_calls"][ph])
            its = stats["pcg_iters_side"][side]
            ipl = its / calls
            avg_s = kms / calls / 1e3
            bpi = stats["pcg_bytes_per_iter"][side]
            kname = ("pcg_mg_kernel" if stats["pcg_multigrid"][side] else
                     "pcg_reg_kernel" if stats["pcg_cluster"][side] else "pcg_grid_kernel")
            sides.append({"side": "uv"[side], "kernel": kname, "kernel_ms_per_step": kms / steps, "launches": calls,
                          "iters": its, "iters_per_launch": ipl, "avg_launch_us": avg_s * 1e6,
                          "us_per_iter": avg_s * 1e6 / max(ipl, 1e-9), "bytes_per_iter": bpi,
                          "achieved": ipl * bpi / avg_s / 1e9 if avg_s > 0 else 0.0,
                          "share_of_step": kms / tot_ms if tot_ms > 0 else None})
        dom = max(sides, key=lambda d: d["kernel_ms_per_step"])
        return {"value": value, "ms_per_step": t_max / steps, "steps": steps, "warmup": warmup,
                "precond": {CR_PRECOND_JACOBI: "jacobi", CR_PRECOND_LEARNED: "learned (flexible CG, Jacobi judge)",
                            CR_PRECOND_MULTIGRID: "multigrid", CR_PRECOND_AUTO: "auto (multigrid on the v side; "
                            "u side multigrid in float64 or above 20,000 rows, else Jacobi)"}[pc],
                "pcg_multigrid_levels": stats["pcg_multigrid"], "time_to_relres_s": ttr,
                "relres_reached_steps": len(reached), "final_relres": infos[-1]["relres"],
                "final_rank": infos[-1]["rank"], "stop": infos[-1]["stop_name"],
                "pcg_iters_per_step": stats["pcg_iters"] / steps,
                "galerkin_cg_iters_per_step": sum(i["cg_iters"] for i in infos) / steps,
                "phase_ms_per_step": {k: v / steps for k, v in stats["phase_ms"].items() if v},
                "gpu_launches": stats["launches"], "clocks": clk.summary(),
                "galerkin_eigen_projections": stats["galerkin_eigen"],
                "pcg": {"dominant": dom, "sides": sides,
                        "share_of_step": pcg_ms / tot_ms if tot_ms > 0 else None,
                        "kernel_share_of_step": kern_ms / tot_ms if tot_ms > 0 else None},
                **({"judge": {"learned_solves": stats["learned_solves"], "fallbacks": stats["learned_fallbacks"],
                              "switched_off_sides": [s for s in (0, 1) if stats["learned_off"] >> s & 1]}}
                   if net is not None else {})}

    forms = {"fp64": measure(CR_FP64), "mixed": measure(CR_MIXED)}
    if not args.no_jacobi and head_pc != CR_PRECOND_JACOBI:
        # the Jacobi-PCG forms beside the headline: what the multigrid preconditioner gains
        jk = min(args.steps, 3)
        forms["fp64_jacobi"] = measure(CR_FP64, steps=jk, warmup=1, precond=CR_PRECOND_JACOBI)
        forms["mixed_jacobi"] = measure(CR_MIXED, steps=jk, warmup=1, precond=CR_PRECOND_JACOBI)
    if not args.no_learned:
        # learned preconditioner: trained once (not timed) on the sub-systems of two
        # other problems of the same family, then the float64 solve with flexible CG
        from paper_1808_05510_gb300 import learned, synth as _synth

        t0 = time.perf_counter()
        train_probs = [_synth.visual_cortex(seed=1900 + k, lam=args.lam, r_max=args.r_max) for k in range(2)]
        t1 = time.perf_counter()
        net, hist, npairs = learned.train_for(train_probs, [0, 5, 10], steps=args.learn_steps, n_random=2, batch=8)
        t2 = time.perf_counter()
        lf = measure(CR_FP64, net=net)
        lf["training"] = {"pairs": npairs, "steps": args.learn_steps, "loss_first": float(np.mean(hist[:10])),
                          "loss_last": float(np.mean(hist[-10:])), "seconds": t2 - t1,
                          "problems": "2 visual-cortex-shaped problems, seeds 1900-1901, ranks 0/5/10, both sides"}
        forms["learned"] = lf
        net.close()
    if not args.no_batch:
        forms["batched"] = measure_batch(args, rank, world, dev, precond=head_pc)
    ttr_toy = None if args.no_ttr else measure_ttr_toy(args)
    ttr_visual = None if args.no_ttr else measure_ttr(p, args, head_pc, r_cap=args.ttr_r, resid_every=args.ttr_resid_every,
                                                      label="visual-cortex workload (7,530 voxels, 28 injections, "
                                                            "lambda 100)")
    cortex = None if args.no_cortex else measure_cortex(args, head_pc)
    post = None if args.no_post else measure_post(p, args, CR_MIXED if args.precision == "mixed" else CR_FP64)
    head = forms[args.precision]
    hbm, peak_kind = peaks()
    dom = head["pcg"]["dominant"]
    roofline = {"bound": "hbm", "achieved": dom["achieved"], "peak": hbm, "unit": "GB/s",
                "frac": dom["achieved"] / hbm,
                "traffic": pcg_traffic(dom["kernel"], args.precision, "uv".index(dom["side"])),
                "kernel": f"{dom['kernel']} ({dom['side']} side, the largest kernel share of the step)",
                "peak_kind": peak_kind, "bytes_per_iter": dom["bytes_per_iter"],
                "kernel_share_of_step": dom["share_of_step"], "pcg_share_of_step": head["pcg"]["share_of_step"],
                "avg_launch_us": dom["avg_launch_us"], "iters_per_launch": dom["iters_per_launch"],
                "us_per_iter": dom["us_per_iter"]}
    out = {"metric": METRIC, "value": head["value"], "unit": UNIT, "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": head["ms_per_step"], "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f32+f64" if args.precision == "mixed" else "f64", "data": "synthetic",
           "config": {**cfg, "residual_every": args.resid_every}, "time_to_relres_s": head["time_to_relres_s"],
           "final_relres": head["final_relres"],
           "final_rank": head["final_rank"], "stop": head["stop"],
           "speedup_vs_fp64": head["value"] / forms["fp64"]["value"],
           "time_to_relres_toy": ttr_toy, "time_to_relres_visual": ttr_visual, "whole_cortex": cortex,
           "postprocess": post,
           "roofline": roofline, "gpu_launches": head["gpu_launches"], "clocks": head["clocks"],
           "forms": {k: {kk: vv for kk, vv in v.items() if kk not in ("clocks",)} for k, v in forms.items()}}
    prec_e2e = CR_MIXED if args.precision == "mixed" else CR_FP64

    # end to end through the public API with host buffers (create + solve + factors + destroy)
    if not args.no_e2e:
        e_ms, e_ranks, h2d, d2h = [], 0, 0, 0
        for k in range(args.steps + 1):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            with ConReg.from_problem(p, r_cap=args.r_max, precision=prec_e2e, precond=head_pc,
                                     residual_every=args.resid_every) as ge:
                info = ge.cr_solve(args.r_max, args.tau, args.relres)
                U, Z, V = ge.cr_get_factors()
                st = ge.cr_get_stats()
            torch.cuda.synchronize()
            el = (time.perf_counter() - t0) * 1e3
            if k == 0:
                continue  # warm-up
            e_ms.append(el)
            e_ranks += info["rank"]
            h2d, d2h = st["h2d_bytes"], st["d2h_bytes"]
        e_r, e_t = replicas.aggregate(e_ranks, sum(e_ms), world, dev)
        out["e2e"] = {"value": e_r / (e_t / 1e3), "unit": UNIT,
                      "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                      "ms_per_step": e_t / args.steps}
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_like_for_like(p, args, prec_e2e, head_pc)
    if rank == 0:
        print(json.dumps(out), flush=True)


def measure_ttr(p, args, precond, r_cap: int, label: str, runs: int = 2, resid_every: int = 1):
    """Time to relative residual 1e-6 (Algorithm 1 from W = 0, stopping at relres <= 1e-6,
    dW <= tau or the rank cap) for the float64 and mixed forms: CUDA events around
    cr_solve on an already created problem (creation untimed), median of `runs`
    after a short warm-up solve."""
    import numpy as np
    import torch

    from paper_1808_05510_gb300.conreg import CR_FP64, CR_MIXED, ConReg

    stream = torch.cuda.current_stream()
    out = {"workload": label, "target": args.relres, "rank_cap": r_cap, "residual_every": resid_every}
    for name, prec in (("fp64", CR_FP64), ("mixed", CR_MIXED)):
        times, info = [], None
        with ConReg.from_problem(p, r_cap=r_cap, precision=prec, precond=precond, residual_every=resid_every,
                                 profile=1) as g:
            g.cr_solve(3, args.tau, args.relres)
            for _ in range(runs):
                g.cr_set_factors(np.zeros((p.ny, 0)), np.zeros((0, 0)), np.zeros((p.nx, 0)))
                g.cr_get_stats(reset=True)
                torch.cuda.synchronize()
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                info = g.cr_solve(r_cap, args.tau, args.relres)
                e1.record(stream)
                e1.synchronize()
                times.append(e0.elapsed_time(e1) / 1e3)
            st = g.cr_get_stats()
        sec = float(np.median(times))
        out[name] = {"seconds": sec, "reached": info["stop_name"] == "relres", "rank": info["rank"],
                     "relres": info["relres"], "stop": info["stop_name"], "updates_per_s": info["rank"] / sec,
                     "pcg_iters": info["pcg_iters"], "galerkin_cg_iters": info["cg_iters"],
                     "phase_ms": {k: round(v, 1) for k, v in st["phase_ms"].items() if v}}
    out["mixed_speedup"] = out["fp64"]["seconds"] / out["mixed"]["seconds"]
    return out


def measure_cortex(args, precond):
    """The whole-cortex-shaped workload (ellipsoidal shell of ~45,000 voxels in a
    96 x 64 x 80 box, 126 injections, lambda 1e3): one greedy solve per form to
    relres 1e-6 or the rank cap, relres checked every few steps."""
    from paper_1808_05510_gb300 import synth as _synth

    t0 = time.perf_counter()
    pc = _synth.whole_cortex()
    gen = time.perf_counter() - t0
    out = measure_ttr(pc, args, precond, r_cap=args.cortex_r, runs=1, resid_every=args.cortex_resid_every,
                      label=f"whole-cortex workload ({pc.ny} voxels in a 96x64x80 shell, {pc.m} injections, "
                            f"lambda {pc.lam:g})")
    out["data_gen_s"] = gen
    return out


def cpu_like_for_like(p, args, prec, precond):
    """The oracle and the GPU on the same work: greedy steps 1..k of the same
    workload from W = 0 (k: what the oracle finishes in --cpu-seconds), residual
    evaluated every step on both sides.  The oracle runs as it stands on all host
    cores and, in a child process limited to one BLAS thread, on one core (its
    first min(k, 2) steps)."""
    import numpy as np
    import torch

    from paper_1808_05510_gb300.conreg import ConReg

    mt = oracle_sample(p, args, args.cpu_seconds)
    k = max(1, mt["steps"])
    st = None
    try:
        env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
        code = ("import json,sys; sys.path.insert(0, %r); import bench; from paper_1808_05510_gb300 import synth; "
                "a = bench.parse_args_list([]); p = synth.visual_cortex(seed=1810, lam=a.lam, r_max=a.r_max); "
                "print(json.dumps(bench.oracle_sample(p, a, %r, max_steps=%d)))" % (ROOT, args.cpu_seconds, min(k, 2)))
        r = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=600)
        st = json.loads(r.stdout.strip().splitlines()[-1])
        st["cores"] = 1
    except Exception as e:  # reported, not fatal
        st = {"error": str(e)[:200]}
    stream = torch.cuda.current_stream()
    with ConReg.from_problem(p, r_cap=max(k, 3), precision=prec, precond=precond) as g:
        g.cr_solve(min(k, 3), args.tau, args.relres)
        g.cr_set_factors(np.zeros((p.ny, 0)), np.zeros((0, 0)), np.zeros((p.nx, 0)))
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        info = g.cr_solve(k, args.tau, args.relres)
        e1.record(stream)
        e1.synchronize()
        gsec = e0.elapsed_time(e1) / 1e3
    mt["single_thread"] = st
    mt["gpu_same_steps"] = {"steps": info["rank"], "seconds": gsec, "value": info["rank"] / gsec,
                            "ratio_to_oracle": (info["rank"] / gsec) / mt["value"] if mt["value"] else None}
    return mt


# float64 FMA throughput of GB300 from its unit counts: 152 SMs x 2 FMA per SM
# per clock x 2 flops x 2.07 GHz (the nominal 1.25 TFLOP/s)
FP64_TFLOPS = 152 * 2 * 2 * 2.07e9 / 1e12


def measure_post(p, args, prec, reps: int = 5):
    """Post-processing of the headline solution at rank r_max: the tiled pass over
    W = U Z V^T with the nonnegative projection (statistics only, W stays on the
    device) and the SVD of the solution, each timed with CUDA events on the
    problem's stream (median of ``reps`` calls after one warm-up)."""
    import torch

    from paper_1808_05510_gb300.conreg import ConReg

    with ConReg.from_problem(p, r_cap=args.r_max, precision=prec) as g:
        g.cr_solve(args.r_max, args.tau, 0.0)
        j = g.cr_get_rank()

        def timed(fn):
            ms = []
            for k in range(reps + 1):
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                torch.cuda.synchronize()
                e0.record(g.stream)
                res = fn()
                e1.record(g.stream)
                e1.synchronize()
                if k:
                    ms.append(e0.elapsed_time(e1))
            return sorted(ms)[len(ms) // 2], res

        rep_ms, rep = timed(lambda: g.cr_solution_report(nonneg=True))
        svd_ms, _ = timed(lambda: g.cr_svd_factors())
    entries = p.ny * p.nx
    flops = 2.0 * entries * j
    achieved = flops / (rep_ms / 1e3) / 1e12
    return {"rank": j, "entries": entries, "report_ms": rep_ms, "svd_ms": svd_ms,
            "entries_per_s": entries / (rep_ms / 1e3), "negative_entries": rep["n_negative"],
            "negative_mass_rms": (rep["neg_fro2"] / entries) ** 0.5,
            "roofline": {"bound": "alu", "achieved": achieved, "peak": FP64_TFLOPS, "unit": "TFLOP/s",
                         "frac": achieved / FP64_TFLOPS, "kernel": "post_tile_kernel (float64 W = U Z V^T tiles)",
                         "peak_kind": "of derived (152 SMs x 2 FP64 FMA/clk x 2.07 GHz)",
                         "flops_per_call": flops}}


def measure_ttr_toy(args, runs: int = 3):
    """Time to relative residual 1e-6 on the toy workload (20 x 20 grid, 5
    injections, lambda = 100), where the greedy reaches it (near rank 90): CUDA
    events around cr_solve from a freshly created problem (creation untimed),
    residual checked every step, median of `runs` after one warm-up."""
    import numpy as np
    import torch
    from paper_1808_05510_gb300 import synth as _synth
    from paper_1808_05510_gb300.conreg import CR_FP64, CR_MIXED, ConReg

    tp = _synth.toy2d()
    stream = torch.cuda.current_stream()
    out = {"workload": "toy 20x20 grid, 5-point Laplacian, 5 injections, lambda 100, rank cap 400",
           "target": 1e-6}
    for name, prec in (("fp64", CR_FP64), ("mixed", CR_MIXED)):
        times, info = [], None
        for k in range(runs + 1):
            with ConReg.from_problem(tp, r_cap=400, precision=prec) as g:
                torch.cuda.synchronize()
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                info = g.cr_solve(400, 1e-13, 1e-6)
                e1.record(stream)
                e1.synchronize()
                if k:
                    times.append(e0.elapsed_time(e1) / 1e3)
        out[name] = {"seconds": float(np.median(times)), "rank": info["rank"], "relres": info["relres"],
                     "stop": info["stop_name"]}
    out["mixed_speedup"] = out["fp64"]["seconds"] / out["mixed"]["seconds"]
    return out


def measure_batch(args, rank=0, world=1, dev="cuda", precond=None):
    """Batched form: the lambda x fold sweep (16 lambdas log-spaced 1..1e6 x 5 folds
    of a 126-injection, ~15,000-voxel data set; every member fits 96-106
    injections) in the mixed form, after the autotuner picked its launch shape.
    Beside it, one member at a time (concurrency 1) on an 8-member sample, every
    other lambda, to show what running members side by side gains.  With
    several ranks every rank solves its shard of the members (weak in GPUs,
    strong in members) and the per-member scores are gathered on the host."""
    import torch
    from paper_1808_05510_gb300 import sweep, synth as _synth
    from paper_1808_05510_gb300.conreg import CR_MIXED, solve_batch

    t0 = time.perf_counter()
    bp = _synth.sweep_cortex()
    folds = _synth.fold_partition(bp.m)
    mem_all = _synth.sweep_members(bp.m, _synth.lambda_grid(), folds)
    mem = replicas.shard_members(mem_all, rank, world)
    gen_s = time.perf_counter() - t0
    pc = {} if precond is None else {"precond": precond}
    solve_batch(bp, mem[:9], r_max=2, tau=args.tau, precision=CR_MIXED, **pc)  # warm-up
    shape = sweep.autotune(bp, mem, r_probe=2, tau=args.tau, precision=CR_MIXED, **pc)
    with ClockSampler(int(os.environ.get("LOCAL_RANK", "0"))) as clk:
        res, sec = sweep._timed_batch(bp, mem, args.batch_r, tau=args.tau, relres_target=args.relres,
                                      concurrency=shape["concurrency"], cluster_size=shape["cluster_size"],
                                      precision=CR_MIXED, **pc)
    ranks, ms_max = replicas.aggregate(sum(r["rank"] for r in res), 1e3 * sec, world, dev)
    sec = ms_max / 1e3
    sample = mem[::max(1, 10 // world)]  # 8 members, every other lambda (fold 0)
    seq, seq_sec = sweep._timed_batch(bp, sample, args.batch_r, tau=args.tau, relres_target=args.relres,
                                      concurrency=1, precision=CR_MIXED, **pc)
    seq_ranks, seq_ms = replicas.aggregate(sum(r["rank"] for r in seq), 1e3 * seq_sec, world, dev)
    seq_sec = seq_ms / 1e3
    # per-member scores of every rank, for the cross-validation curve
    scored = [(m, r) for part in replicas.gather_objects(list(zip(mem, res)), world) for m, r in part]
    cv = sweep.cv_summary([m for m, _ in scored], [r for _, r in scored])
    res = [r for _, r in scored]
    status = {}
    for r in res:
        status[str(r["status"])] = status.get(str(r["status"]), 0) + 1
    torch.cuda.synchronize()
    return {"value": ranks / sec, "unit": UNIT + " (aggregate over members)", "seconds": sec,
            "members": len(mem_all), "members_per_rank": len(mem), "voxels": bp.nx, "ninj_total": bp.m,
            "ninj_fit": sorted({len(f) for _, f, _ in mem}), "r_max": args.batch_r, "precision": "mixed",
            "ranks": ranks, "shape": {k: shape[k] for k in ("concurrency", "cluster_size")},
            "autotune": shape["table"], "status_counts": status,
            "sequential_sample": {"members": len(sample) * world, "seconds": seq_sec, "value": seq_ranks / seq_sec},
            "speedup_vs_sequential": (ranks / sec) / (seq_ranks / seq_sec),
            "pcg_iters": sum(r["pcg_iters"] for r in res), "galerkin_cg_iters": sum(r["cg_iters"] for r in res),
            "best_lambda": cv["best_lambda"], "cv_by_lambda": {f"{k:.3g}": v for k, v in cv["cv_by_lambda"].items()},
            "final_relres_range": [min(r["relres"] for r in res), max(r["relres"] for r in res)],
            "data_gen_s": gen_s, "clocks": clk.summary()}


def main():
    args = parse()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    if world > 1:
        import torch
        import torch.distributed as dist

        torch.cuda.set_device(local_rank)
        dist.init_process_group("nccl")
    try:
        run_ours(args, rank, world, local_rank)
    finally:
        if world > 1:
            import torch.distributed as dist

            dist.destroy_process_group()


if __name__ == "__main__":
    main()
