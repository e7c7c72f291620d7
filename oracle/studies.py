"""Spectrum and epsilon-rank studies on the paper's own workload (oracle side).

Test infrastructure (see ``oracle/__init__``).

The §4.1 setup: N points from the standard normal distribution in d
dimensions, x_c at the origin; the n points closest to the origin are the
sources S, rho = their largest norm, and the targets are the points at
distance >= xi rho from x_c (xi = 1). K = K(T, S) with the Gaussian kernel
(§4.2, eq. eqn_gaussian_kernel); h is given in units of Silverman's h_S
(eq. eqn_silverman_bandwidth).

* ``far_spectrum``: the singular values of K (§4.2.2, "Singular values of
  K"); the epsilon-rank is the smallest r with sigma_{r+1} / sigma_1 < eps
  (§4.1.3 step 1). Reading: the singular values are the square roots of the
  eigenvalues of K^T K (LAPACK's symmetric eigensolver as a library step);
  that resolves every sigma_k >= 1e-7 sigma_1, far below the eps = 1e-2 of
  the paper's studies.
* ``bandwidth_for_rank``: the bandwidth search of Table 2: for a rank budget
  kappa (a fraction of n), bisection in log h for the h where the eps-rank
  crosses kappa n, on the small-h side (the rank grows with h) or on the
  large-h side (the rank falls with h). Reading: the search window and the
  number of bisection steps are parameters (the paper gives neither); the
  result is the window's midpoint after the last step.
* ``interaction_fractions``: Table 3's Self, NN and Far fractions
  ||K_*||_2 / ||K||_2 of the N x n matrix of all points (sources included)
  against the sources (eq. eqn_interation_splits): K_S the n sources, K_N
  the next n points by distance to the origin, K_F the remaining N - 2n.
"""
from __future__ import annotations

import numpy as np

from .kernels import silverman_bandwidth


def paper_shape(d: int, N: int = 100000, n: int = 500, seed: int = 0, xi: float = 1.0):
    """(points sorted by distance to the origin (ties to the lower index), rho, far-field mask, h_S)."""
    from workloads import standard_normal
    X = standard_normal(N, d, seed=seed)
    X = X[np.argsort(np.sum(X * X, axis=1), kind="stable")]
    rho = float(np.sqrt(np.max(np.sum(X[:n] * X[:n], axis=1))))
    far = np.sum(X * X, axis=1) >= (xi * rho) ** 2
    far[:n] = False
    return X, rho, far, silverman_bandwidth(d, N)


def _gram(Y, S, h, chunk=16384):
    """K^T K for K = exp(-||y - x||^2 / (2 h^2)) over targets Y and sources S, by row chunks.

    The squared distances come from ||y||^2 + ||x||^2 - 2 y.x (a library matrix product as a step),
    clamped at zero: on this unit-scale data their rounding error is about 1e-14, far below what the
    eps = 1e-2 rank or the 2-norm ratios can see."""
    S = np.asarray(S, dtype=np.float64)
    s2 = np.sum(S * S, axis=1)
    G = np.zeros((S.shape[0], S.shape[0]))
    for a in range(0, Y.shape[0], chunk):
        Yc = Y[a:a + chunk]
        D2 = np.maximum(np.sum(Yc * Yc, axis=1)[:, None] + s2[None, :] - 2.0 * (Yc @ S.T), 0.0)
        B = np.exp(-D2 / (2.0 * h * h))
        G += B.T @ B
    return G


def far_spectrum(X, n, far, h):
    """Singular values (decreasing) of K(far targets, sources) at bandwidth h."""
    ev = np.linalg.eigvalsh(_gram(X[far], X[:n], h))[::-1]
    return np.sqrt(np.maximum(ev, 0.0))


def eps_rank_of(sv, eps):
    """Smallest r with sv[r] / sv[0] < eps (sv decreasing)."""
    sv = np.asarray(sv)
    if sv.size == 0 or sv[0] <= 0.0:
        return 0
    small = np.flatnonzero(sv / sv[0] < eps)
    return int(small[0]) if small.size else int(sv.size)


def bandwidth_for_rank(X, n, far, h_S, kappa, side, eps=1e-2, lo=None, hi=None, steps=20):
    """h / h_S where the eps-rank of K(far, sources) crosses round(kappa n); side -1: small h, +1: large h."""
    target = int(round(kappa * n))
    if lo is None or hi is None:
        lo, hi = (1.0, 20.0) if side > 0 else (0.01, 1.0)
    a, b = np.log(lo), np.log(hi)
    for _ in range(steps):
        m = 0.5 * (a + b)
        r = eps_rank_of(far_spectrum(X, n, far, np.exp(m) * h_S), eps)
        if (side > 0 and r > target) or (side < 0 and r < target):
            a = m
        else:
            b = m
    return float(np.exp(0.5 * (a + b)))


def interaction_fractions(X, n, h):
    """(Self, NN, Far) = ||K_S||_2, ||K_N||_2, ||K_F||_2 over ||K||_2, K = K(all points, sources)."""
    S = X[:n]
    GS, GN, GF = _gram(X[:n], S, h), _gram(X[n:2 * n], S, h), _gram(X[2 * n:], S, h)
    norm = lambda G: float(np.sqrt(max(np.linalg.eigvalsh(G)[-1], 0.0)))   # noqa: E731
    tot = norm(GS + GN + GF)
    return norm(GS) / tot, norm(GN) / tot, norm(GF) / tot
