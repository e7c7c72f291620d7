"""Interpolative decomposition from the pivoted QR, and its error (oracle side).

Test infrastructure (see ``oracle/__init__``).

Definition (§2.1.3, "Interpolative Decomposition"): K ~ C P with C = r columns
of K (the skeleton) and P (r x n) containing the r x r identity. Appendix A.1:
with K Pi = Q [R11 R12; 0 R22] and R11 of size r x r, P solves R11 P = R12
and the skeleton is the first r pivots. R11 is square and, while the pivots
are nonzero, nonsingular, so that system has the unique solution
T = R11^-1 R12, found here by back-substitution.

Output convention shared with the CUDA path:
  skel_perm[0:r]  skeleton columns in pivot order;
  skel_perm[r:n]  the other columns in ascending index order;
  T (r x (n-r))   K(:, skel_perm[r+c]) ~ sum_i T[i, c] K(:, skel_perm[i]);
  P = [I_r  T] Pi^T assembled on demand by ``assemble_P``.
"""
from __future__ import annotations

import math

import numpy as np

from .cpqr import cpqr
from .kernels import LAPLACE, kernel_block, squared_distances


def back_substitution(R11, B):
    """Solve R11 X = B for upper-triangular R11, one row at a time from the bottom."""
    r = R11.shape[0]
    X = np.zeros((r, B.shape[1]), dtype=np.float64)
    for i in range(r - 1, -1, -1):
        acc = B[i] - R11[i, i + 1:] @ X[i + 1:]
        X[i] = acc / R11[i, i]
    return X


def interpolative_decomposition(K, r_max, tol=0.0):
    """ID of K (s x n) at fixed rank r_max (tol <= 0) or at relative tolerance tol.

    Returns dict(skel_perm, T, rank, r22_rel, qr).
    """
    K = np.asarray(K, dtype=np.float64)
    n = K.shape[1]
    qr = cpqr(K, r_max, tol)
    A, piv, r = qr["A"], qr["piv"], qr["rank"]
    mask = np.ones(n, dtype=bool)
    mask[piv] = False
    rest = np.flatnonzero(mask)
    R11 = np.zeros((r, r), dtype=np.float64)
    for k in range(r):
        R11[:k + 1, k] = A[:k + 1, piv[k]]
    R12 = A[:r, rest]
    T = back_substitution(R11, R12) if r > 0 else np.zeros((0, rest.size))
    r22_rel = qr["r22"] / qr["fro"] if qr["fro"] > 0 else 0.0
    return {"skel_perm": np.concatenate([piv, rest]).astype(np.int64), "T": T,
            "rank": r, "r22_rel": r22_rel, "qr": qr}


def assemble_P(skel_perm, T, n):
    """P (r x n) with P[:, skel_perm[:r]] = I_r and P[:, skel_perm[r:]] = T."""
    r = T.shape[0]
    P = np.zeros((r, n), dtype=np.float64)
    P[np.arange(r), skel_perm[:r]] = 1.0
    P[:, skel_perm[r:]] = T
    return P


def _fsum_squares(E, chunk=1 << 16):
    flat = np.asarray(E, dtype=np.float64).reshape(-1)
    return math.fsum(float(np.sum(flat[a:a + chunk] ** 2)) for a in range(0, flat.size, chunk))


def reconstruction_error(K, skel_perm, T):
    """||K - K(:,J) P||_F / ||K||_F; skeleton columns are reproduced exactly."""
    K = np.asarray(K, dtype=np.float64)
    r = T.shape[0]
    J, rest = skel_perm[:r], skel_perm[r:]
    E = K[:, rest] - K[:, J] @ T
    num = _fsum_squares(E)
    den = _fsum_squares(K)
    return math.sqrt(num / den) if den > 0 else 0.0


def full_block_error(kernel, Y_far, X_node, skel_perm, T, row_chunk=4096):
    """Relative Frobenius error of the ID on the full far-field block (§4.1.3 step 4).

    K is evaluated in row chunks over all far-field targets; each chunk's
    residual K(:, rest) - K(:, J) T is accumulated in exactly rounded sums.
    The Laplace block is evaluated unscaled per chunk relative to one common
    scale (the smallest distance over the whole block), so the ratio is exact.
    """
    Y_far = np.asarray(Y_far, dtype=np.float64)
    r = T.shape[0]
    J, rest = skel_perm[:r], skel_perm[r:]
    num_parts, den_parts = [], []
    if kernel.kind == LAPLACE:  # one scale for the whole block
        d = Y_far.shape[1]
        ln_rmin = min(0.5 * math.log(float(squared_distances(Y_far[a:a + row_chunk], X_node).min()))
                      for a in range(0, Y_far.shape[0], row_chunk))
    for a in range(0, Y_far.shape[0], row_chunk):
        Yc = Y_far[a:a + row_chunk]
        if kernel.kind == LAPLACE:
            Kc = np.exp(-(d - 2) * (0.5 * np.log(squared_distances(Yc, X_node)) - ln_rmin))
        else:
            Kc, _ = kernel_block(kernel, Yc, X_node)
        E = Kc[:, rest] - Kc[:, J] @ T
        num_parts.append(_fsum_squares(E))
        den_parts.append(_fsum_squares(Kc))
    den = math.fsum(den_parts)
    return math.sqrt(math.fsum(num_parts) / den) if den > 0 else 0.0
