"""The paper's other row samplers for the sampled block (oracle side).

Test infrastructure (see ``oracle/__init__``).

§4.1.3 compares, beside uniform sampling, three ways to pick the s rows of the
sampled block from the far field T of a source set S with centre x_c:

* distance sampling: rows drawn without replacement with probability
  proportional to the distance from the target to x_c (§4.1.3's list); the
  heuristic of §3 argues for probabilities inversely proportional to the
  distance from the sources, and the experiments are read here as that
  (both are provided: ``inverse`` selects);
* leverage sampling: probability proportional to the row's leverage score
  (§3, Def. "Statistical Leverage"), which needs the full block;
* nearest neighbours: deterministically the s targets closest to the source
  points, distance to the nearest source (ties to the lower row index).

Draws without replacement use Efraimidis & Spirakis' keys ln(u_i) / w_i
(Inf. Proc. Letters 97, 2006) with u_i the unit double of draw i (i = the
candidate's position) of stream (seed, stream_id, DOMAIN_PAPER_SAMPLERS); the s
largest keys win, ties to the lower position, rows in decreasing key order.
"""
from __future__ import annotations

import numpy as np

from .philox import DOMAIN_PAPER_SAMPLERS, draws, to_unit_double
from .spectral import eps_rank, row_leverage_scores


def weighted_draw(candidates, w, s, seed, stream_id):
    """s candidates without replacement with probabilities proportional to w > 0 (in key order)."""
    candidates = np.asarray(candidates, dtype=np.int64)
    w = np.asarray(w, dtype=np.float64)
    u = to_unit_double(draws(seed, stream_id, DOMAIN_PAPER_SAMPLERS, 0, candidates.size))
    keys = np.log(u) / w
    order = np.lexsort((np.arange(candidates.size), -keys))
    return candidates[order[:min(int(s), candidates.size)]], keys


def distance_weights(Y, candidates, x_c, inverse=True):
    """||y - x_c|| (§4.1.3's list) or its inverse (§3's heuristic) for the candidate targets."""
    y = np.asarray(Y, dtype=np.float64)[np.asarray(candidates, dtype=np.int64)]
    r = np.sqrt(np.sum((y - np.asarray(x_c, dtype=np.float64)) ** 2, axis=1))
    return 1.0 / r if inverse else r


def distance_sample(Y, candidates, x_c, s, seed, stream_id, inverse=True):
    return weighted_draw(candidates, distance_weights(Y, candidates, x_c, inverse), s, seed, stream_id)[0]


def leverage_sample(K, candidates, s, eps, seed, stream_id):
    """Rows of the full far-field block K (one per candidate, same order) drawn by leverage at the eps-rank."""
    r = eps_rank(K, eps)
    if r == 0:
        return np.asarray(candidates, dtype=np.int64)[:0]
    lev = row_leverage_scores(K, r)
    keep = lev > 0.0
    return weighted_draw(np.asarray(candidates, dtype=np.int64)[keep], lev[keep], s, seed, stream_id)[0]


def nearest_neighbours(Y, candidates, X, s):
    """The s candidate targets closest to the source points (distance to the nearest source)."""
    candidates = np.asarray(candidates, dtype=np.int64)
    y = np.asarray(Y, dtype=np.float64)[candidates]
    X = np.asarray(X, dtype=np.float64)
    dmin = np.full(candidates.size, np.inf)
    for j in range(X.shape[0]):
        dmin = np.minimum(dmin, np.sum((y - X[j]) ** 2, axis=1))
    order = np.lexsort((candidates, dmin))
    return candidates[order[:min(int(s), candidates.size)]]
