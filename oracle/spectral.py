"""Truncated-SVD error, epsilon-rank, leverage scores and coherence (oracle side).

Test infrastructure (see ``oracle/__init__``). The singular values come from
LAPACK (numpy.linalg.svd), used as a library step.

* Truncated SVD (§2.1.3): the best rank-r approximation has spectral error
  sigma_{r+1} and Frobenius error sqrt(sum_{k>r} sigma_k^2) (the paper prints
  the Frobenius form without the squares and root; the squared form is the
  correct one).
* epsilon-rank (§4.1.3 step 1): the smallest r with sigma_{r+1}/sigma_1 < eps.
* Leverage (§3, Def. "Statistical Leverage"): for A = K^T the scores are the
  squared row norms of V_r; for the m x n block K that is the squared row
  norms of U_r, one score per target row. They sum to r and lie in [0, 1];
  the coherence gamma is their maximum, r/m <= gamma <= 1 (eq. gamma_def).
"""
from __future__ import annotations

import numpy as np


def singular_values(K):
    return np.linalg.svd(np.asarray(K, dtype=np.float64), compute_uv=False)


def svd_frobenius_error(K, r: int) -> float:
    sv = singular_values(K)
    tot = float(np.sum(sv * sv))
    return float(np.sqrt(np.sum(sv[r:] ** 2) / tot)) if tot > 0 else 0.0


def svd_spectral_error(K, r: int) -> float:
    sv = singular_values(K)
    return float(sv[r] / sv[0]) if r < sv.size else 0.0


def eps_rank(K, eps: float) -> int:
    sv = singular_values(K)
    if sv.size == 0 or sv[0] == 0.0:
        return 0
    small = np.flatnonzero(sv / sv[0] < eps)
    return int(small[0]) if small.size else int(sv.size)


def row_leverage_scores(K, r: int) -> np.ndarray:
    U, _, _ = np.linalg.svd(np.asarray(K, dtype=np.float64), full_matrices=False)
    Ur = U[:, :r]
    return np.sum(Ur * Ur, axis=1)


def coherence(K, r: int) -> float:
    return float(np.max(row_leverage_scores(K, r)))
