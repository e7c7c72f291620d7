"""Seeded synthetic point sets for the far-field compression workloads.

This module only draws input points. It holds none of the method's arithmetic
(no sampling of kernel rows, no kernel evaluation, no factorisation), so both
the CUDA path's tests/benchmarks and the CPU oracle may use it to obtain the
same inputs.

Every generator uses numpy's PCG64 stream seeded by ``seed``; the stream is
platform independent, so x86 and Arm hosts produce bit-identical points.

Workloads (sizes of the paper's experiments, §4.1, and of the benchmark suite):

* ``single_block``      512 sources uniform in [0,1]^4, 2,048 targets with the
                        first coordinate uniform in [3,4] and the rest in [0,1].
* ``gaussian_mixture``  N points from an equal-weight mixture of isotropic
                        Gaussians (means uniform in [-5,5]^d, sigma = 1), the
                        d=16 tree-compression workload.
* ``decaying_mixture``  d=128 mixture whose per-coordinate variance decays as 1/k.
* ``low_intrinsic``     intrinsic dimension d_i normal data embedded in d_e
                        dimensions by a random orthonormal map plus small
                        Gaussian noise (§4.1.1 "Low intrinsic dimension").
* ``standard_normal``   the §4.1.1 "Normal" data set.

Workload parameter: ``median_pairwise_distance`` gives the Gaussian bandwidth
of the d = 1000 workload (the exact median over all pairs of the first 4,096
points).

Random inputs of the learned proposal (drawn here so both sides share them):

* ``mlp_init``          initial FP32 parameters of the 12-128-128-1 network
                        (flat vector; layout in ``MLP_LAYOUT``).
* ``projections``       the 8 random directions g_k ~ N(0, I/d) of the
                        projection features.
"""
from __future__ import annotations

import numpy as np

__all__ = [
    "single_block",
    "gaussian_mixture",
    "decaying_mixture",
    "low_intrinsic",
    "standard_normal",
    "random_matrix",
    "mlp_init",
    "projections",
    "median_pairwise_distance",
    "MLP_LAYOUT",
    "MLP_N_PARAMS",
]


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(int(seed)))


def single_block(seed: int = 0, n: int = 512, m: int = 2048, d: int = 4):
    """Sources X (n x d) uniform in [0,1]^d; targets Y (m x d) with y_0 in [3,4].

    The targets are well separated from the sources along the first axis, so
    the whole target set is the far field of the source box.
    Returns (X, Y) as float64 row-major arrays.
    """
    g = _rng(seed)
    X = g.random((n, d))
    Y = g.random((m, d))
    Y[:, 0] += 3.0
    return np.ascontiguousarray(X), np.ascontiguousarray(Y)


def gaussian_mixture(N: int = 65536, d: int = 16, k: int = 8, seed: int = 0,
                     mean_range: float = 5.0, sigma: float = 1.0) -> np.ndarray:
    """Equal-weight mixture of k isotropic Gaussians; means uniform in [-r, r]^d."""
    g = _rng(seed)
    means = g.uniform(-mean_range, mean_range, size=(k, d))
    comp = g.integers(0, k, size=N)
    X = means[comp] + sigma * g.standard_normal((N, d))
    return np.ascontiguousarray(X)


def decaying_mixture(N: int = 262144, d: int = 128, k: int = 16, seed: int = 0,
                     mean_range: float = 5.0) -> np.ndarray:
    """Mixture of k Gaussians whose coordinate-k variance is 1/k (k = 1..d).

    Means are uniform in [-mean_range, mean_range] scaled by 1/sqrt(k) per
    coordinate, so both the spread of the means and the within-component
    variance decay along the coordinates.
    """
    g = _rng(seed)
    scale = 1.0 / np.sqrt(np.arange(1, d + 1, dtype=np.float64))
    means = g.uniform(-mean_range, mean_range, size=(k, d)) * scale
    comp = g.integers(0, k, size=N)
    X = means[comp] + g.standard_normal((N, d)) * scale
    return np.ascontiguousarray(X)


def low_intrinsic(N: int = 100000, d_i: int = 10, d_e: int = 1000, noise: float = 0.01,
                  seed: int = 0, dtype=np.float32) -> np.ndarray:
    """x = Q z + noise, z ~ N(0, I_{d_i}), Q a seeded random d_e x d_i orthonormal map."""
    g = _rng(seed)
    G = g.standard_normal((d_e, d_i))
    Q, _ = np.linalg.qr(G)
    Z = g.standard_normal((N, d_i))
    X = Z @ Q.T + noise * g.standard_normal((N, d_e))
    return np.ascontiguousarray(X.astype(dtype))


def standard_normal(N: int, d: int, seed: int = 0) -> np.ndarray:
    """N points from the d-dimensional standard normal distribution."""
    return np.ascontiguousarray(_rng(seed).standard_normal((N, d)))


def random_matrix(m: int, n: int, seed: int = 0, decay: float | None = None) -> np.ndarray:
    """Dense m x n test matrix; with ``decay`` its singular values fall as decay**k."""
    g = _rng(seed)
    if decay is None:
        return g.standard_normal((m, n))
    k = min(m, n)
    U, _ = np.linalg.qr(g.standard_normal((m, k)))
    V, _ = np.linalg.qr(g.standard_normal((n, k)))
    sv = decay ** np.arange(k, dtype=np.float64)
    return (U * sv) @ V.T


# Flat parameter vector of the proposal network (FP32 master copy): name ->
# (offset, shape). Matrices are row-major with W[j, k] = weight from input k
# to unit j. This is an interface shared by value, not code: each side of the
# project spells it out itself.
MLP_LAYOUT = {
    "W1": (0, (128, 12)),
    "b1": (1536, (128,)),
    "W2": (1664, (128, 128)),
    "b2": (18048, (128,)),
    "w3": (18176, (128,)),
    "b3": (18304, (1,)),
}
MLP_N_PARAMS = 18305


def mlp_init(seed: int = 0) -> np.ndarray:
    """He-normal initial weights (std sqrt(2 / fan_in)), zero biases, as float32.

    The output layer uses std sqrt(1 / fan_in) / 4 so that the initial logits
    are small and the initial proposal is close to uniform.
    """
    g = _rng(seed)
    theta = np.zeros(MLP_N_PARAMS, dtype=np.float64)
    for name, fan_in, std in (("W1", 12, np.sqrt(2.0 / 12)), ("W2", 128, np.sqrt(2.0 / 128)),
                              ("w3", 128, 0.25 * np.sqrt(1.0 / 128))):
        off, shape = MLP_LAYOUT[name]
        size = int(np.prod(shape))
        theta[off:off + size] = std * g.standard_normal(size)
    return theta.astype(np.float32)


def projections(d: int, seed: int = 0, k: int = 8) -> np.ndarray:
    """k x d matrix of independent N(0, 1/d) entries (float64)."""
    return np.ascontiguousarray(_rng(seed).standard_normal((k, d)) / np.sqrt(d))


def median_pairwise_distance(points: np.ndarray, k: int = 4096) -> float:
    """Exact median of ||x_i - x_j|| over all pairs i < j of the first k points."""
    S = np.asarray(points[:k], dtype=np.float64)
    sq = np.sum(S * S, axis=1)
    D2 = np.maximum(sq[:, None] + sq[None, :] - 2.0 * (S @ S.T), 0.0)
    iu = np.triu_indices(S.shape[0], 1)
    return float(np.median(np.sqrt(D2[iu])))
