"""Pins of the paper's other samplers (§4.1.3): distance, leverage, nearest neighbours."""
import numpy as np
from scipy.spatial.distance import cdist

import workloads
from oracle import kernels as o_kernels
from oracle import samplers
from oracle import spectral


def _chi2(counts, p):
    n = counts.sum()
    expect = n * p
    return float(np.sum((counts - expect) ** 2 / expect))


def test_weighted_draw_single_draw_probabilities():
    w = np.array([0.5, 1.0, 2.0, 4.0, 0.25, 1.5])
    cand = np.arange(10, 16)
    counts = np.zeros(6)
    for sid in range(4000):
        rows, _ = samplers.weighted_draw(cand, w, 1, 3, sid)
        counts[rows[0] - 10] += 1
    assert _chi2(counts, w / w.sum()) < 25.0      # 5 d.o.f.: P(chi2 > 25) < 2e-4


def test_weighted_draw_structure_and_prefix():
    g = np.random.default_rng(1)
    cand = g.choice(1000, 60, replace=False)
    w = g.random(60) + 0.1
    small, keys = samplers.weighted_draw(cand, w, 10, 5, 9)
    big, _ = samplers.weighted_draw(cand, w, 30, 5, 9)
    assert np.unique(big).size == 30 and list(big[:10]) == list(small)
    pos = {int(c): i for i, c in enumerate(cand)}
    k = keys[[pos[int(c)] for c in big]]
    assert np.all(np.diff(k) <= 0)


def test_distance_weights_closed_form():
    Y = np.array([[3.0, 4.0], [0.0, 2.0], [1.0, 1.0]])
    x_c = np.array([0.0, 0.0])
    np.testing.assert_allclose(samplers.distance_weights(Y, [0, 1, 2], x_c, inverse=False), [5.0, 2.0, np.sqrt(2)])
    np.testing.assert_allclose(samplers.distance_weights(Y, [0, 1, 2], x_c), [0.2, 0.5, 1 / np.sqrt(2)])


def test_nearest_neighbours_match_a_library_distance_matrix():
    X, Y = workloads.single_block(2, n=40, m=300)
    cand = np.arange(300)
    nn = samplers.nearest_neighbours(Y, cand, X, 25)
    dmin = cdist(Y, X, "sqeuclidean").min(axis=1)
    assert list(nn) == list(np.lexsort((cand, dmin))[:25])


def test_leverage_sample_draws_by_the_leverage_scores():
    K = workloads.random_matrix(12, 5, seed=4, decay=0.5)
    lev = spectral.row_leverage_scores(K, spectral.eps_rank(K, 1e-12))
    counts = np.zeros(12)
    for sid in range(4000):
        rows = samplers.leverage_sample(K, np.arange(12), 1, 1e-12, 7, sid)
        counts[rows[0]] += 1
    assert _chi2(counts, lev / lev.sum()) < 40.0   # 11 d.o.f.: P(chi2 > 40) < 1e-4


def test_far_field_of_a_gaussian_block_favours_near_rows_under_inverse_distance():
    X, Y = workloads.single_block(0)
    x_c = X.mean(axis=0)
    w_inv = samplers.distance_weights(Y, np.arange(Y.shape[0]), x_c)
    K, _ = o_kernels.kernel_block(o_kernels.Kernel(o_kernels.GAUSSIAN, h=1.0), Y, X)
    row_norm = np.linalg.norm(K, axis=1)
    # the heuristic of §3: near rows carry the largest norms, and get the largest inverse-distance weights
    assert np.corrcoef(w_inv, row_norm)[0, 1] > 0.5
