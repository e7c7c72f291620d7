"""Spectrum and epsilon-rank studies of the far field on the GPU (§4.1 setup, §4.2 Tables 2 and 3).

The workload is the paper's: N points from the standard normal distribution, x_c at the origin,
the n points closest to it as the sources, rho their largest norm, the targets at distance >= xi rho.
Every heavy step runs in libffc: the nearest points to the origin (ffc_sample_paper, nearest
neighbours of a single source at x_c), the far field (ffc_far_field), the Gaussian blocks
(ffc_eval_block, FP64) and their singular values and eps-rank (ffc_spectrum: Gram matrix and Jacobi
eigenvalues, FP64). This module only orders the points and runs the searches.

* ``far_spectrum(h)``: singular values of K(targets, sources) and the eps-rank (smallest r with
  sigma_{r+1} / sigma_1 < eps).
* ``bandwidth_for_rank``: Table 2's search, bisection in log h for the h where the eps-rank crosses
  kappa n, on the small-h side (the rank grows with h) or the large-h side (it falls with h).
* ``interaction_fractions``: Table 3's ||K_S||_2, ||K_N||_2, ||K_F||_2 over ||K||_2 for the N x n
  matrix of all points against the sources: K_S the sources, K_N the next n points by distance to
  the origin, K_F the rest.
"""
from __future__ import annotations

import math

import torch

from . import ffc


def silverman_bandwidth(d: int, N: int) -> float:
    """h_S = (4 / (2 d + 1))^(1 / (d + 4)) N^(-1 / (d + 4)) (§4.2.1, eq. eqn_silverman_bandwidth)."""
    return (4.0 / (2 * d + 1)) ** (1.0 / (d + 4)) * N ** (-1.0 / (d + 4))


class PaperShape:
    """The §4.1 workload on the device: points reordered so that the n sources come first (nearest to
    the origin, in order), then the next n (their nearest neighbours), then the rest."""

    def __init__(self, X: torch.Tensor, n: int = 500, xi: float = 1.0):
        ffc._dev(X, "X")
        N, d = X.shape
        self.N, self.d, self.n, self.xi = N, d, n, xi
        origin = torch.zeros((1, d), dtype=X.dtype, device=X.device)
        cand = torch.arange(N, dtype=torch.int64, device=X.device)
        near = ffc.ffc_sample_paper(ffc.DRAW_NEAREST, X, cand, 2 * n, 0, 0, X=origin)   # 2n nearest, in order
        rest = torch.ones(N, dtype=torch.bool, device=X.device)
        rest[near] = False
        self.X = X[torch.cat([near, torch.nonzero(rest).flatten()])].contiguous()
        self.rho = float(torch.linalg.vector_norm(self.X[n - 1].double()))
        self.x_c = torch.zeros(d, dtype=torch.float64, device=X.device)
        self.far = ffc.ffc_far_field(self.X, x_c=self.x_c, radius=self.rho, xi=xi, ex_begin=0, ex_end=n)
        self.h_S = silverman_bandwidth(d, N)

    def block(self, rows: torch.Tensor, h: float) -> torch.Tensor:
        """Column-major storage (n x len(rows)) of the FP64 Gaussian block K(X[rows], sources)."""
        K, _ = ffc.ffc_eval_block(ffc.Kernel(ffc.GAUSSIAN, h=h), self.X, rows, self.X[: self.n])
        return K.t()

    def far_spectrum(self, h: float, eps: float = 1e-2):
        """(singular values (decreasing), eps-rank) of K(far field, sources) at bandwidth h."""
        sigma, r, _ = ffc.ffc_spectrum(self.block(self.far, h), eps)
        return sigma, r

    def bandwidth_for_rank(self, kappa: float, side: int, eps: float = 1e-2, lo=None, hi=None, steps: int = 20):
        """h / h_S where the eps-rank crosses round(kappa n); side -1: small h, +1: large h."""
        target = int(round(kappa * self.n))
        if lo is None or hi is None:
            lo, hi = (1.0, 20.0) if side > 0 else (0.01, 1.0)
        a, b = math.log(lo), math.log(hi)
        for _ in range(steps):
            m = 0.5 * (a + b)
            _, r = self.far_spectrum(math.exp(m) * self.h_S, eps)
            if (side > 0 and r > target) or (side < 0 and r < target):
                a = m
            else:
                b = m
        return math.exp(0.5 * (a + b))

    def interaction_fractions(self, h: float):
        """(Self, NN, Far) fractions of ||K||_2 (Table 3)."""
        n, N = self.n, self.N
        idx = torch.arange(N, dtype=torch.int64, device=self.X.device)
        norm = lambda rows: float(ffc.ffc_spectrum(self.block(rows, h), 0.0)[0][0])   # noqa: E731
        tot = norm(idx)
        return norm(idx[:n]) / tot, norm(idx[n:2 * n]) / tot, norm(idx[2 * n:]) / tot
