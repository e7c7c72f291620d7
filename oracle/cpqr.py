"""Businger-Golub column-pivoted Householder QR in FP64 (oracle side).

Test infrastructure (see ``oracle/__init__``).

The ID is computed from a rank-revealing QR K Pi = Q R (§2.1.3, ID theorem;
Appendix A.1 step 2). This is the classical greedy form: at step k the pivot
is the remaining column of largest residual norm; a Householder reflector
zeroes it below row k and is applied to every remaining column.

Readings (the paper is silent on these details):

* residual column norms are recomputed exactly at every step (no downdating);
* ties in the pivot norm go to the smallest original column index;
* the reflector follows LAPACK dlarfg: beta = -sign(alpha) * ||x|| with
  sign(0) = +1, tau = (beta - alpha) / beta, v = x / (alpha - beta), v_0 = 1;
  when x has no component below its first entry, H = I and beta = alpha;
* columns are never moved: the factorisation marks selected columns, so the
  returned array holds R in the original column positions;
* stopping: with tol > 0 the rank is the smallest k <= r_max with
  ||R22(k)||_F <= tol * ||K||_F, where ||R22(k)||_F^2 is the sum of the
  residual column norms after k steps; with tol <= 0 the rank is r_max. The
  loop also stops when every remaining column is exactly zero.
"""
from __future__ import annotations

import math

import numpy as np


def householder(x):
    """LAPACK-dlarfg reflector for vector x: returns (v, tau, beta)."""
    x = np.asarray(x, dtype=np.float64)
    alpha = float(x[0])
    xnorm = float(np.sqrt(np.sum(x[1:] * x[1:]))) if x.size > 1 else 0.0
    v = np.zeros_like(x)
    v[0] = 1.0
    if xnorm == 0.0:
        return v, 0.0, alpha
    norm = math.hypot(alpha, xnorm)
    beta = -norm if alpha >= 0.0 else norm
    tau = (beta - alpha) / beta
    v[1:] = x[1:] / (alpha - beta)
    return v, tau, beta


def cpqr(K, r_max, tol=0.0):
    """Column-pivoted QR of K (s x n).

    Returns a dict with
      A      the factored array: for a selected column p_k, A[:k, p_k] is the
             part of R11 above the diagonal and A[k, p_k] = beta_k; for an
             unselected column j, A[:r, j] is R12 and A[r:, j] is R22;
      piv    the selected columns in pivot order (length r);
      rank   r;
      r22    ||R22(r)||_F;
      fro    ||K||_F;
      norms  the residual column norms at each step (list of arrays, for tests).
    """
    A = np.array(K, dtype=np.float64, copy=True)
    s, n = A.shape
    fro = float(np.sqrt(np.sum(A * A)))
    selected = np.zeros(n, dtype=bool)
    piv: list[int] = []
    kmax = min(int(r_max), s, n)
    r22 = fro
    for k in range(kmax + 1):
        free = np.flatnonzero(~selected)
        norms2 = np.sum(A[k:, free] * A[k:, free], axis=0) if k < s else np.zeros(free.size)
        r22 = float(np.sqrt(np.sum(norms2)))
        if tol > 0.0 and r22 <= tol * fro:
            break
        if k == kmax or free.size == 0:
            break
        best = int(np.argmax(norms2))          # first maximum = lowest index
        if norms2[best] == 0.0:
            break
        p = int(free[best])
        v, tau, beta = householder(A[k:, p])
        rest = free[free != p]
        w = v @ A[k:, rest]
        A[k:, rest] -= tau * np.outer(v, w)
        A[k, p] = beta
        A[k + 1:, p] = 0.0
        selected[p] = True
        piv.append(p)
    return {"A": A, "piv": np.asarray(piv, dtype=np.int64), "rank": len(piv),
            "r22": r22, "fro": fro}
