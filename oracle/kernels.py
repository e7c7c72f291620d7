"""Kernel functions and kernel-block evaluation in FP64 (oracle side).

Test infrastructure (see ``oracle/__init__``).

K_ij = K(y_i, x_j): rows are targets, columns are sources (eq. e:sum, §1).

* Gaussian   K(y,x) = exp(-||x - y||^2 / (2 h^2))             (§4.2, eq. gaussian_kernel)
* Laplace    K(y,x) = ||x - y||^(2-d), d != 2                  (§4.3)
* Polynomial K(y,x) = (x^T y / h + c)^p                        (§4.4)

Distances are formed from direct coordinate differences. The Laplace block is
returned scaled by its largest entry: K_ij = exp(-(d-2) (ln r_ij - ln r_min)),
with ln(scale) = -(d-2) ln r_min returned beside it. A scalar multiple of the
block changes neither the pivoted QR's pivots nor R11^-1 R12 nor any relative
error, and it keeps d = 128 entries (about 10^-150 unscaled) in range.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

GAUSSIAN, LAPLACE, POLYNOMIAL = 0, 1, 2


@dataclass(frozen=True)
class Kernel:
    kind: int
    h: float = 1.0
    c: float = 1.0
    p: int = 3


class KernelDomainError(ValueError):
    """Raised for a singular Laplace block (coincident points) or d == 2."""


def squared_distances(Y, X, row_chunk=256):
    """D2_ij = sum_k (y_ik - x_jk)^2 from direct differences."""
    Y = np.asarray(Y, dtype=np.float64)
    X = np.asarray(X, dtype=np.float64)
    D2 = np.empty((Y.shape[0], X.shape[0]), dtype=np.float64)
    for a in range(0, Y.shape[0], row_chunk):
        diff = Y[a:a + row_chunk, None, :] - X[None, :, :]
        D2[a:a + row_chunk] = np.sum(diff * diff, axis=2)
    return D2


def kernel_block(kernel: Kernel, Y, X):
    """Evaluate the m x n block K(Y, X). Returns (K, log_scale)."""
    Y = np.asarray(Y, dtype=np.float64)
    X = np.asarray(X, dtype=np.float64)
    if kernel.kind == GAUSSIAN:
        D2 = squared_distances(Y, X)
        return np.exp(-D2 / (2.0 * kernel.h * kernel.h)), 0.0
    if kernel.kind == LAPLACE:
        d = Y.shape[1]
        if d == 2:
            raise KernelDomainError("the d = 2 (logarithmic) Laplace kernel is not supported")
        D2 = squared_distances(Y, X)
        if D2.size == 0:
            return D2, 0.0
        if np.any(D2 == 0.0):
            raise KernelDomainError("coincident source and target: Laplace kernel is singular")
        ln_r = 0.5 * np.log(D2)
        ln_rmin = float(ln_r.min())
        K = np.exp(-(d - 2) * (ln_r - ln_rmin))
        return K, -(d - 2) * ln_rmin
    if kernel.kind == POLYNOMIAL:
        G = Y @ X.T
        return (G / kernel.h + kernel.c) ** kernel.p, 0.0
    raise ValueError(f"unknown kernel kind {kernel.kind}")


def kernel_value(kernel: Kernel, y, x) -> float:
    """Unscaled scalar K(y, x), written straight from the paper's formulas."""
    y = np.asarray(y, dtype=np.float64)
    x = np.asarray(x, dtype=np.float64)
    if kernel.kind == GAUSSIAN:
        return float(np.exp(-np.sum((x - y) ** 2) / (2.0 * kernel.h ** 2)))
    if kernel.kind == LAPLACE:
        d = y.shape[0]
        return float(np.sqrt(np.sum((x - y) ** 2)) ** (2 - d))
    if kernel.kind == POLYNOMIAL:
        return float((np.dot(x, y) / kernel.h + kernel.c) ** kernel.p)
    raise ValueError(kernel.kind)


def silverman_bandwidth(d: int, N: int) -> float:
    """h_S = (4 / (2d + 1))^(1/(d+4)) N^(-1/(d+4))  (§4.2.1, eq. silverman_bandwidth)."""
    return (4.0 / (2.0 * d + 1.0)) ** (1.0 / (d + 4.0)) * N ** (-1.0 / (d + 4.0))
