"""Host logic of the lambda x fold sweep (sweep.py) on the CPU: the autotuner's
probe selection and choice of launch shape with the timed batch replaced by a
fake of known cost, and the cross-validation summary against a hand-computed
curve."""
import math

import numpy as np
import pytest

from paper_1808_05510_gb300 import sweep


def members(lams, n_folds=2):
    return [(lam, np.arange(3), np.arange(3, 5)) for lam in lams for _ in range(n_folds)]


@pytest.fixture
def fake_batch(monkeypatch):
    calls = []

    def fake(p, mem, r_max, **kw):
        calls.append({"members": list(mem), "r_max": r_max, **kw})
        # a made-up cost: 16-CTA clusters better, concurrency 18 best
        conc, cs = kw["concurrency"], kw["cluster_size"]
        rate = (1.0 if cs == 16 else 0.4) * (1.0 - abs(conc - 18) / 40.0)
        ranks = r_max * len(mem)
        return [{"rank": r_max} for _ in mem], ranks / rate / 100.0

    monkeypatch.setattr(sweep, "_timed_batch", fake)
    return calls


def test_autotune_picks_the_fastest_shape_on_the_costliest_members(fake_batch):
    lams = [10.0 ** k for k in range(8)]
    mem = members(lams, n_folds=5)  # 40 members
    shape = sweep.autotune(None, mem, r_probe=3, tau=1e-7, galerkin_ctas=8)
    assert (shape["concurrency"], shape["cluster_size"]) == (18, 16)
    assert len(shape["table"]) == len(sweep.DEFAULT_CANDIDATES)
    # the probe is the 2 x max-concurrency largest-lambda members (here all 40 are fewer than 72)
    n_probe = min(len(mem), 2 * max(c for c, _ in sweep.DEFAULT_CANDIDATES))
    assert shape["probe_members"] == n_probe == 40
    for c in fake_batch:
        assert c["r_max"] == 3 and c["tau"] == 1e-7 and c["galerkin_ctas"] == 8
        probe_lams = [m[0] for m in c["members"]]
        assert probe_lams == sorted(probe_lams, reverse=True)
    best = max(shape["table"], key=lambda t: t["ranks_per_s"])
    assert best["concurrency"] == 18 and best["cluster_size"] == 16


def test_autotune_probe_takes_the_largest_lambdas(fake_batch):
    lams = [10.0 ** k for k in range(8)]
    mem = members(lams, n_folds=5)
    sweep.autotune(None, mem, r_probe=1, candidates=((4, 16), (8, 16)), probe_members=6)
    for c in fake_batch:
        assert [m[0] for m in c["members"]] == [1e7] * 5 + [1e6]


def test_cv_summary_by_hand():
    mem = members([1.0, 10.0, 100.0], n_folds=2)
    res = [{"cv_num": n, "cv_den": d} for n, d in [(1, 4), (3, 4), (1, 8), (1, 8), (2, 2), (2, 2)]]
    out = sweep.cv_summary(mem, res)
    assert out["cv_by_lambda"] == {1.0: 0.5, 10.0: 0.125, 100.0: 1.0}
    assert out["best_lambda"] == 10.0
    # a lambda whose folds hold no observed held-out entries has no score and is
    # never the best, wherever it sorts
    out = sweep.cv_summary(members([5.0], 1), [{"cv_num": 0.0, "cv_den": 0.0}])
    assert math.isnan(out["cv_by_lambda"][5.0]) and out["best_lambda"] is None
    out = sweep.cv_summary(members([0.5, 5.0], 1), [{"cv_num": 0.0, "cv_den": 0.0}, {"cv_num": 3.0, "cv_den": 4.0}])
    assert math.isnan(out["cv_by_lambda"][0.5]) and out["best_lambda"] == 5.0


def test_cv_summary_sets_aside_unconverged_members():
    """A lambda with a fold that stopped at an iteration cap (CR_ENOTCONV) is
    counted and not chosen while some lambda has all folds converged."""
    mem = members([1.0, 10.0], n_folds=2)
    res = [{"cv_num": n, "cv_den": d, "status": s} for n, d, s in [(1, 4, 0), (1, 4, 0), (1, 8, 4), (1, 8, 0)]]
    out = sweep.cv_summary(mem, res)
    assert out["cv_by_lambda"] == {1.0: 0.25, 10.0: 0.125}
    assert out["not_converged"] == {1.0: 0, 10.0: 1}
    assert out["best_lambda"] == 1.0 and out["best_lambda_all_converged"]
    # every lambda has an unconverged fold: the plain minimum, flagged
    res[0]["status"] = 4
    out = sweep.cv_summary(mem, res)
    assert out["best_lambda"] == 10.0 and not out["best_lambda_all_converged"]
