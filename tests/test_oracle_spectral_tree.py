"""Pins for the oracle's spectral helpers, tree and per-node compression."""
import math

import numpy as np
import pytest

import workloads
from oracle import compress, interp, kernels, spectral, tree
from oracle.kernels import GAUSSIAN, Kernel
from oracle.sampling import far_field_mask


def _known_svd(m, n, sv, seed=0):
    g = np.random.default_rng(seed)
    U, _ = np.linalg.qr(g.standard_normal((m, len(sv))))
    V, _ = np.linalg.qr(g.standard_normal((n, len(sv))))
    return U, (U * sv) @ V.T


def test_eps_rank_and_truncated_svd_error_closed_form():
    sv = np.array([1.0, 0.5, 0.1, 1e-3, 1e-7, 1e-9])
    _, K = _known_svd(30, 20, sv)
    assert spectral.eps_rank(K, 1e-2) == 3       # sigma_4/sigma_1 = 1e-3 < 1e-2
    assert spectral.eps_rank(K, 1e-6) == 4
    want = math.sqrt(np.sum(sv[3:] ** 2) / np.sum(sv ** 2))
    assert spectral.svd_frobenius_error(K, 3) == pytest.approx(want, rel=1e-8)
    assert spectral.svd_spectral_error(K, 2) == pytest.approx(0.1, rel=1e-10)


def test_leverage_scores_closed_form_and_coherence_bounds():
    sv = np.array([3.0, 2.0, 1.0, 0.5])
    U, K = _known_svd(50, 10, sv, seed=4)
    for r in (1, 2, 3):
        lev = spectral.row_leverage_scores(K, r)
        np.testing.assert_allclose(lev, np.sum(U[:, :r] ** 2, axis=1), atol=1e-12)
        assert lev.sum() == pytest.approx(r, rel=1e-12)
        assert lev.min() >= -1e-15 and lev.max() <= 1 + 1e-12
        gamma = spectral.coherence(K, r)
        assert r / 50 - 1e-12 <= gamma <= 1 + 1e-12


def test_tree_depth_and_layout():
    assert tree.tree_depth(65536, 256) == 8
    assert tree.tree_depth(100000, 512) == 8
    assert tree.tree_depth(262144, 256) == 10
    b, c, lv = tree.node_layout(100000, 8)
    leaves = c[lv == 8]
    assert set(leaves.tolist()) == {390, 391} and leaves.sum() == 100000
    assert c[lv == 2].tolist() == [25000] * 4


def test_principal_direction_matches_top_eigenvector():
    g = np.random.default_rng(0)
    C = g.standard_normal((500, 6)) * np.array([5.0, 1, 1, 1, 1, 1])
    C = C @ np.linalg.qr(g.standard_normal((6, 6)))[0]
    C -= C.mean(0)
    v = tree.principal_direction(C)
    w, V = np.linalg.eigh(C.T @ C)
    top = V[:, -1]
    assert abs(abs(v @ top) - 1.0) < 1e-12
    assert v[np.argmax(np.abs(v))] > 0


def test_tree_invariants():
    X = workloads.gaussian_mixture(N=3000, d=5, k=4, seed=2)
    t = tree.build_tree(X, 100)
    assert t.depth == 5
    assert sorted(t.perm.tolist()) == list(range(3000))
    for i in range(t.n_nodes):
        b, c = int(t.begin[i]), int(t.count[i])
        P = X[t.perm[b:b + c]]
        np.testing.assert_allclose(t.centroid[i], P.mean(0), atol=1e-12)
        assert t.radius[i] == pytest.approx(np.sqrt(((P - t.centroid[i]) ** 2).sum(1)).max(), rel=1e-12)
        if t.level[i] < t.depth:
            # the split separates the two halves along the node's principal direction
            C = P - t.centroid[i]
            v = tree.principal_direction(C)
            pl, pr = C[: c // 2] @ v, C[c // 2:] @ v
            assert pl.max() <= pr.min()


def test_compress_small_tree_contract():
    X = workloads.gaussian_mixture(N=4096, d=4, k=4, seed=1)
    t = tree.build_tree(X, 256)
    Xp = X[t.perm]
    k = Kernel(GAUSSIAN, h=1.0)
    res = compress.compress_tree(Xp, t, k, tol=1e-6, seed=0, s0=32, s_max=512,
                                 nodes=[3, 4, 9, 20])
    for nr in res:
        b, c = int(t.begin[nr.node]), int(t.count[nr.node])
        far = far_field_mask(Xp, t.centroid[nr.node], t.radius[nr.node], 1.0, b, b + c)
        assert far[nr.rows].all() and len(set(nr.rows.tolist())) == nr.s
        assert nr.far_count == int(far.sum())
        if nr.status == compress.STATUS_OK:
            assert nr.r22_rel <= 1e-6
            all_rows = nr.s < nr.attempts[-1]
            assert nr.rank <= compress.rank_cap(nr.s, c, all_rows, 256)
        # the reported ID reproduces the sampled block to ||R22||
        K, _ = kernels.kernel_block(k, Xp[nr.rows], Xp[b:b + c])
        assert interp.reconstruction_error(K, nr.skel_perm, nr.T) == pytest.approx(nr.r22_rel, rel=1e-6, abs=1e-15)
        # every earlier attempt was a prefix of the final sample
        assert nr.attempts == [32 * 2 ** i for i in range(len(nr.attempts))]
