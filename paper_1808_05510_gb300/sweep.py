"""Lambda x fold sweep on top of ``cr_solve_batch``: the autotuner that picks
its launch shape, and the cross-validation summary.

The tunable shape of a sweep is how the GPU's SMs are shared between member
solves: how many members run at once (``concurrency``) and how many CTAs tile
one member's PCG vectors (the thread-block ``cluster_size``: 16 CTAs give each
member more SMs, 8 CTAs let twice as many members run side by side).  The
autotuner times a short probe of the actual sweep -- the costliest members
(largest lambda) for ``r_probe`` greedy steps -- for every candidate shape and
keeps the one with the most rank-1 updates per second.  All arithmetic runs in
the library; this module only times calls and aggregates their results.
"""
from __future__ import annotations

import itertools
import math
import time
from typing import Dict, List, Optional, Sequence, Tuple

import numpy as np

from . import conreg

# (concurrency, cluster_size): 16-CTA clusters won every probe so far, so the
# 8-CTA shape keeps two candidates and the search spends its time on concurrency
DEFAULT_CANDIDATES: Tuple[Tuple[int, int], ...] = tuple(
    itertools.product((9, 18, 27, 36), (16,))) + ((18, 8), (36, 8))


def _timed_batch(p, members, r_max, **kw):
    import torch

    stream = torch.cuda.current_stream()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    res = conreg.solve_batch(p, members, r_max=r_max, stream=stream, **kw)
    e1.record(stream)
    e1.synchronize()
    return res, e0.elapsed_time(e1) / 1e3


def autotune(p, members, r_probe: int = 2, candidates: Sequence[Tuple[int, int]] = DEFAULT_CANDIDATES,
             probe_members: Optional[int] = None, tau: float = 1e-9, **opts) -> Dict:
    """Time every (concurrency, cluster_size) candidate on a probe of the sweep and
    return {"concurrency", "cluster_size", "table": [...]} for the fastest.  The
    probe takes the 2 x max-concurrency costliest members (largest lambda)."""
    order = sorted(range(len(members)), key=lambda k: -members[k][0])
    n_probe = probe_members or min(len(members), 2 * max(c for c, _ in candidates))
    probe = [members[k] for k in order[:n_probe]]
    table = []
    for conc, cs in candidates:
        res, sec = _timed_batch(p, probe, r_probe, tau=tau, concurrency=conc, cluster_size=cs, **opts)
        ranks = sum(r["rank"] for r in res)
        table.append({"concurrency": conc, "cluster_size": cs, "seconds": sec,
                      "ranks_per_s": ranks / sec if sec > 0 else 0.0})
    best = max(table, key=lambda t: t["ranks_per_s"])
    return {"concurrency": best["concurrency"], "cluster_size": best["cluster_size"], "probe_members": n_probe,
            "r_probe": r_probe, "table": table}


CR_ENOTCONV = 4  # cr_status of a member whose solve stopped at an iteration cap


def cv_summary(members, results) -> Dict:
    """Mean held-out error per lambda over its folds (sum of numerators over sum
    of denominators) and the lambda that minimises it.

    A member whose solve stopped at an iteration cap (status CR_ENOTCONV) is
    scored on an unconverged iterate: ``not_converged`` counts them per lambda,
    and a lambda with any such fold is left out of the choice of
    ``best_lambda`` unless no lambda has all its folds converged."""
    per: Dict[float, List[float]] = {}
    nc: Dict[float, int] = {}
    for (lam, _, _), r in zip(members, results):
        a = per.setdefault(lam, [0.0, 0.0])
        a[0] += r["cv_num"]
        a[1] += r["cv_den"]
        nc[lam] = nc.get(lam, 0) + (1 if r.get("status", 0) == CR_ENOTCONV else 0)
    curve = {lam: (v[0] / v[1] if v[1] > 0 else float("nan")) for lam, v in sorted(per.items())}
    scored = [lam for lam, e in curve.items() if not math.isnan(e)]  # NaN: no observed held-out entry
    clean = [lam for lam in scored if nc[lam] == 0]
    pool = clean if clean else scored
    best = min(pool, key=lambda lam: curve[lam]) if pool else None
    return {"cv_by_lambda": curve, "best_lambda": best,
            "not_converged": {lam: nc[lam] for lam in sorted(nc)},
            "best_lambda_all_converged": bool(clean)}


def run(p, members, r_max: int, tau: float = 1e-9, tune: bool = True, **opts) -> Dict:
    """Autotune (optional), then the timed sweep; returns results, seconds, shape and CV summary."""
    shape = autotune(p, members, tau=tau, **opts) if tune else {"concurrency": 0, "cluster_size": 0}
    t0 = time.perf_counter()
    res, sec = _timed_batch(p, members, r_max, tau=tau, concurrency=shape["concurrency"],
                            cluster_size=shape["cluster_size"], **opts)
    wall = time.perf_counter() - t0
    return {"results": res, "seconds": sec, "wall_seconds": wall, "shape": shape, **cv_summary(members, res)}
