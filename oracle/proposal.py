"""Learned row proposal: features, weighted sampling, leverage targets (oracle side).

Test infrastructure (see ``oracle/__init__``).

The paper ranks row distributions for the sampled block (§4.1.3: uniform,
distance, leverage, nearest neighbours) and finds leverage sampling the most
reliable (§4.2-4.4), but the leverage scores (§3, Def. "Statistical
Leverage") need a basis of the full far-field block. The learned proposal
predicts them from cheap per-row features and samples with them.

Readings used here (the paper has no learned part):

* Features of a candidate target y for a node with centroid x_c and radius
  rho, with delta = y - x_c and r = ||delta|| (12 values):
    f0 = r / rho
    f1 = K(y, x_c) normalised to at most 1 in the far field:
         Gaussian exp(-r^2 / (2 h^2)); Laplace (rho / r)^(d-2);
         polynomial (y.x_c / h + c)^p / (||y|| ||x_c|| / h + c)^p
    f2 = ||y|| / rho
    f3 = rho / h  (h = 1 for the Laplace kernel, which has no length scale)
    f4..f11 = <g_k, delta> / rho for the 8 given random directions g_k.
  A node with rho = 0 uses rho = 1.
* Candidate pool: the whole far field in ascending index order (the
  leverage distribution of §3 is over every row of the block, and the rows
  that carry it are few: a uniform pool of a few times s rows misses them).
  Optionally a uniform pool of a fixed number P of rows (the uniform sampler
  with s = P, same stream) bounds the cost. The pool does not depend on s.
* The network gives a logit o_i per pool row (FP16 weights, FP64 arithmetic
  here); weights w_i = exp(o_i - max o);
  mixed weights w'_i = 0.9 w_i / mean(w) + 0.1, so every row keeps at least
  a tenth of its uniform weight. s rows are drawn without replacement with
  probabilities proportional to w' by Efraimidis & Spirakis' keys (Inf. Proc.
  Letters 97, 2006): key_i = ln(u_i) / w'_i, u_i the unit double of draw i
  (i = pool position) of stream (seed, stream_id, DOMAIN_WEIGHTED_KEYS); the
  s largest keys win, ties to the lower pool position, rows in decreasing key
  order (the whole pool when it has at most s rows). The keys do not depend
  on s, so a size-s sample is a prefix of the size-2s sample.
* Training targets: the leverage scores of the node's full far-field block K
  (m x n) with respect to its epsilon-rank r (§4.1.3 step 1), divided by r
  so they sum to one over the node's rows (sum_i l_i = r, §3).
"""
from __future__ import annotations

import numpy as np

from .kernels import GAUSSIAN, LAPLACE, POLYNOMIAL, Kernel
from .mlp import forward, half_weights
from .philox import DOMAIN_WEIGHTED_KEYS, draws, to_unit_double
from .sampling import far_field_mask, sample_uniform_from_mask
from .spectral import eps_rank, row_leverage_scores

N_FEATURES = 12
UNIFORM_MIX = 0.1


def features(Y, rows, x_c, rho, kernel: Kernel, proj):
    """R x 12 feature rows of the targets Y[rows]."""
    Y = np.asarray(Y, dtype=np.float64)
    y = Y[np.asarray(rows, dtype=np.int64)]
    x_c = np.asarray(x_c, dtype=np.float64)
    proj = np.asarray(proj, dtype=np.float64)
    d = Y.shape[1]
    rho = float(rho) if rho > 0 else 1.0
    delta = y - x_c[None, :]
    r = np.sqrt(np.sum(delta * delta, axis=1))
    ynorm = np.sqrt(np.sum(y * y, axis=1))
    if kernel.kind == GAUSSIAN:
        kc = np.exp(-(r * r) / (2.0 * kernel.h * kernel.h))
        h = kernel.h
    elif kernel.kind == LAPLACE:
        kc = (rho / r) ** (d - 2)
        h = 1.0
    elif kernel.kind == POLYNOMIAL:
        xn = float(np.sqrt(np.sum(x_c * x_c)))
        kc = ((y @ x_c) / kernel.h + kernel.c) ** kernel.p / ((ynorm * xn) / kernel.h + kernel.c) ** kernel.p
        h = kernel.h
    else:
        raise ValueError(kernel.kind)
    F = np.empty((y.shape[0], N_FEATURES), dtype=np.float64)
    F[:, 0] = r / rho
    F[:, 1] = kc
    F[:, 2] = ynorm / rho
    F[:, 3] = rho / h
    F[:, 4:12] = (delta @ proj.T) / rho
    return F


def mixed_weights(o):
    """w' = 0.9 w / mean(w) + 0.1 with w = exp(o - max o)."""
    o = np.asarray(o, dtype=np.float64)
    w = np.exp(o - np.max(o))
    return (1.0 - UNIFORM_MIX) * w / np.mean(w) + UNIFORM_MIX


def es_keys(wp, seed, stream_id):
    """Efraimidis-Spirakis keys ln(u_i) / w'_i for pool positions 0..P-1."""
    u = to_unit_double(draws(seed, stream_id, DOMAIN_WEIGHTED_KEYS, 0, len(wp)))
    return np.log(u) / np.asarray(wp, dtype=np.float64)


def weighted_select(pool_rows, o, s, seed, stream_id):
    """s pool rows without replacement, probability proportional to w'(o).

    Returns (rows in decreasing key order, keys of the whole pool).
    """
    pool_rows = np.asarray(pool_rows, dtype=np.int64)
    P = pool_rows.size
    keys = es_keys(mixed_weights(o), seed, stream_id)
    order = np.lexsort((np.arange(P), -keys))      # key descending, then position
    return pool_rows[order[:min(int(s), P)]], keys


def candidate_pool(far, seed, stream_id, pool_rows: int = 0):
    """The whole far field (pool_rows = 0) or a uniform pool of pool_rows rows."""
    if pool_rows <= 0:
        return np.flatnonzero(far)
    return sample_uniform_from_mask(far, int(pool_rows), seed, stream_id)


def propose_from_mask(far, Y, s, seed, stream_id, x_c, rho, kernel: Kernel, proj, theta32,
                      pool_rows: int = 0):
    """Learned proposal of s far-field rows (far = boolean far-field mask)."""
    pool = candidate_pool(far, seed, stream_id, pool_rows)
    if pool.size == 0:
        return pool
    F = features(Y, pool, x_c, rho, kernel, proj)
    o, _ = forward(half_weights(theta32), F)
    rows, _ = weighted_select(pool, o, s, seed, stream_id)
    return rows


def propose_rows(Y, s, seed, stream_id, x_c, radius, kernel: Kernel, proj, theta32, xi=1.0,
                 ex_begin=0, ex_end=0, pool_rows: int = 0):
    """Returns (rows, far_count) for the far field of (x_c, radius, xi) minus [ex_begin, ex_end)."""
    far = far_field_mask(Y, x_c, radius, xi, ex_begin, ex_end)
    return propose_from_mask(far, Y, s, seed, stream_id, x_c, radius, kernel, proj, theta32,
                             pool_rows), int(far.sum())


def leverage_targets(K, eps):
    """(l / r, r): leverage scores of K's rows at its eps-rank r, normalised to sum 1."""
    r = eps_rank(K, eps)
    if r == 0:
        return np.zeros(np.asarray(K).shape[0]), 0
    lev = row_leverage_scores(K, r)
    return lev / r, r
