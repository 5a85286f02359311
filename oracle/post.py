"""CPU float64 oracle for the post-processing of a greedy solution W = U Z V^T.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import or call this
module: only the tests, ``__graft_entry__.smoke()`` and the CPU legs of
``bench.py`` use it.  It shares no code with the CUDA library.  Every function
forms W densely and applies the definition directly:

* Sec. 4 (leading singular vectors of the solution): W = U Z V^T is not an SVD
  because Z is not diagonal; with the SVD of the core, Z = U~ S V~^T, the
  factors U^ = U U~ and V^ = V V~ give the SVD W = U^ S V^^T.  numpy's SVD of Z
  serves as one step.
* Sec. 3 (error measures): the RMS error E(W, W*) = |W - W*|_F / sqrt(ny nx)
  and the relative error E_rel(W, W*) = |W - W*|_F / |W*|_F.
* Sec. 4 (dropping the nonnegativity constraint): the projection of W onto the
  nonnegative orthant, (W_proj)_ik = max(0, W_ik), and the count and size of
  the negative entries of W.

Readings where the paper is silent: singular values are returned in
descending order; the reference solution W* of a report is given in the same
factored form (U*, Z*, V*) with any rank, W* = 0 at rank 0; the projection,
when asked for, is applied to W before it is compared with W*.
"""
from __future__ import annotations

import math
from typing import Dict, Optional, Tuple

import numpy as np


def dense_w(U, Z, V) -> np.ndarray:
    """W = U Z V^T (ny x nx); the zero matrix at rank 0."""
    U = np.asarray(U, dtype=np.float64)
    V = np.asarray(V, dtype=np.float64)
    if U.shape[1] == 0:
        return np.zeros((U.shape[0], V.shape[0]))
    return U @ np.asarray(Z, dtype=np.float64) @ V.T


def solution_svd(U, Z, V) -> Tuple[np.ndarray, np.ndarray, np.ndarray]:
    """Sec. 4: (U^, sigma, V^) with Z = U~ diag(sigma) V~^T, U^ = U U~, V^ = V V~,
    sigma descending, so that W = U^ diag(sigma) V^^T."""
    Ut, s, Vth = np.linalg.svd(np.asarray(Z, dtype=np.float64))
    return np.asarray(U) @ Ut, s, np.asarray(V) @ Vth.T


def rms_error(W, Wref) -> float:
    """Sec. 3: E(W, W*) = |W - W*|_F / sqrt(ny nx)."""
    W = np.asarray(W)
    return float(np.linalg.norm(W - Wref) / math.sqrt(W.size))


def rel_error(W, Wref) -> float:
    """Sec. 3: E_rel(W, W*) = |W - W*|_F / |W*|_F."""
    return float(np.linalg.norm(np.asarray(W) - Wref) / np.linalg.norm(Wref))


def project_nonneg(W) -> np.ndarray:
    """Sec. 4: the entrywise projection max(0, W) onto the nonnegative orthant."""
    return np.maximum(np.asarray(W, dtype=np.float64), 0.0)


def solution_report(U, Z, V, nonneg: bool = False, ref: Optional[Tuple] = None) -> Dict:
    """Statistics of W = U Z V^T and of its distance to a reference W* = U* Z* V*^T.

    About W itself: ``n_negative`` (entries below zero), ``w_min``, ``w_max``,
    ``w_fro2`` = |W|_F^2 and ``neg_fro2`` = |W - max(0, W)|_F^2.  About the
    compared matrix P(W) (P = max(0, .) if ``nonneg`` else the identity):
    ``ref_fro2`` = |W*|_F^2, ``diff_fro2`` = |P(W) - W*|_F^2, ``diff_maxabs`` =
    max |P(W) - W*|, and the Sec. 3 measures ``rms`` = sqrt(diff_fro2 / (ny nx))
    and ``rel`` = sqrt(diff_fro2 / ref_fro2) (NaN when W* = 0).  ``W_out`` is P(W)."""
    W = dense_w(U, Z, V)
    Wref = np.zeros_like(W) if ref is None else dense_w(*ref)
    PW = project_nonneg(W) if nonneg else W
    D = PW - Wref
    neg = W[W < 0.0]
    diff2 = float(np.sum(D * D))
    ref2 = float(np.sum(Wref * Wref))
    return {
        "entries": int(W.size),
        "n_negative": int(neg.size),
        "w_min": float(W.min()) if W.size else 0.0,
        "w_max": float(W.max()) if W.size else 0.0,
        "w_fro2": float(np.sum(W * W)),
        "neg_fro2": float(np.sum(neg * neg)),
        "ref_fro2": ref2,
        "diff_fro2": diff2,
        "diff_maxabs": float(np.abs(D).max()) if D.size else 0.0,
        "rms": math.sqrt(diff2 / W.size) if W.size else 0.0,
        "rel": math.sqrt(diff2 / ref2) if ref2 > 0.0 else float("nan"),
        "W_out": PW,
    }
