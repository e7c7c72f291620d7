"""Pins of the outgoing-representation oracle (§2.1.3: q~ = P q, u ~ C q~).

* A full-rank ID (r = n) represents the block exactly, so C q~ is K q.
* For any ID, |K q - C P q| <= ||K - C P||_2 ||q|| <= ||K - C P||_F ||q||.
* Low-rank blocks: with a polynomial kernel of exact rank C(d + p, p), the
  representation at that rank reproduces K q to rounding.
"""
import math

import numpy as np

import workloads
from oracle import apply as o_apply
from oracle import interp as o_interp
from oracle import kernels as o_kernels


def _id(K, r_max, tol=0.0):
    ref = o_interp.interpolative_decomposition(K, r_max, tol)
    return ref["skel_perm"], ref["T"], ref["rank"]


def test_full_rank_representation_is_exact():
    X, Y = workloads.single_block(0, n=64, m=200)
    k = o_kernels.Kernel(o_kernels.GAUSSIAN, h=1.0)
    K, _ = o_kernels.kernel_block(k, Y, X)
    skel, T, r = _id(K, 64)
    assert r == 64 and T.shape == (64, 0)
    q = np.random.default_rng(1).standard_normal(64)
    qt = o_apply.skeleton_charges(skel, T, q)
    assert np.array_equal(qt, q[skel[:64]])
    u, _ = o_apply.direct_potential(k, Y, X, q)
    ut, _ = o_apply.id_potential(k, Y, X, skel, r, qt)
    assert np.max(np.abs(u - ut)) <= 1e-12 * np.max(np.abs(u))


def test_error_within_the_block_error_times_the_charges():
    X, Y = workloads.single_block(0)
    k = o_kernels.Kernel(o_kernels.GAUSSIAN, h=1.0)
    K, _ = o_kernels.kernel_block(k, Y, X)
    g = np.random.default_rng(2)
    for r_max in (8, 32, 64):
        skel, T, r = _id(K, r_max)
        P = o_interp.assemble_P(skel, T, K.shape[1])
        E = K - K[:, skel[:r]] @ P
        for _ in range(3):
            q = g.standard_normal(K.shape[1])
            qt = o_apply.skeleton_charges(skel, T, q)
            u, _ = o_apply.direct_potential(k, Y, X, q)
            ut, _ = o_apply.id_potential(k, Y, X, skel, r, qt)
            err = np.linalg.norm(u - ut)
            assert err <= np.linalg.norm(E, 2) * np.linalg.norm(q) * (1 + 1e-9) + 1e-12
            assert err <= np.linalg.norm(E) * np.linalg.norm(q) * (1 + 1e-9) + 1e-12


def test_polynomial_exact_rank_reproduces_the_potential():
    d, p = 3, 2
    g = np.random.default_rng(3)
    X = g.standard_normal((40, d))
    Y = g.standard_normal((90, d))
    k = o_kernels.Kernel(o_kernels.POLYNOMIAL, h=2.0, c=1.0, p=p)
    K, _ = o_kernels.kernel_block(k, Y, X)
    rank = math.comb(d + p, p)
    skel, T, r = _id(K, rank)
    q = g.standard_normal(40)
    u, _ = o_apply.direct_potential(k, Y, X, q)
    ut, _ = o_apply.id_potential(k, Y, X, skel, r, o_apply.skeleton_charges(skel, T, q))
    assert r == rank
    assert np.max(np.abs(u - ut)) <= 1e-9 * np.max(np.abs(u))


def test_laplace_potentials_share_the_scale():
    X, Y = workloads.single_block(1, n=48, m=120, d=5)
    Y = Y + 2.0
    k = o_kernels.Kernel(o_kernels.LAPLACE)
    K, _ = o_kernels.kernel_block(k, Y, X)
    skel, T, r = _id(K, 48)
    q = np.random.default_rng(4).standard_normal(48)
    u, lu = o_apply.direct_potential(k, Y, X, q)
    ut, lt = o_apply.id_potential(k, Y, X, skel, r, o_apply.skeleton_charges(skel, T, q))
    assert lu == lt
    assert np.max(np.abs(u - ut)) <= 1e-10 * np.max(np.abs(u))


# ---------------------------------------------------------------- the tree evaluation

import pytest  # noqa: E402

from oracle import tree as o_tree  # noqa: E402
from oracle.sampling import far_field_mask  # noqa: E402


def _small_tree(seed=5, N=1500, d=3, leaf=48):
    P = workloads.gaussian_mixture(N=N, d=d, k=3, seed=seed)
    t = o_tree.build_tree(P, leaf)
    return P[t.perm], t


_KERNELS = [o_kernels.Kernel(o_kernels.GAUSSIAN, h=0.8), o_kernels.Kernel(o_kernels.LAPLACE),
            o_kernels.Kernel(o_kernels.POLYNOMIAL, h=3.0, c=1.0, p=2)]


@pytest.mark.parametrize("kernel", _KERNELS, ids=["gaussian", "laplace", "polynomial"])
def test_tree_direct_far_plus_near_is_the_all_pairs_sum(kernel):
    """Interaction lists plus near leaves count every source other than the target exactly once:
    the direct-mode tree evaluation equals sum_{j != i} K(x_i, x_j) q_j."""
    Xp, t = _small_tree()
    q = np.random.default_rng(6).standard_normal(len(Xp))
    u_tree = o_apply.tree_potential(kernel, Xp, t, q, mode="direct")
    u_all = o_apply.direct_sum_without_self(kernel, Xp, q)
    assert np.max(np.abs(u_tree - u_all)) <= 1e-11 * np.max(np.abs(u_all))
    # the far part alone is a proper subset: the near field carries the rest
    u_far = o_apply.tree_potential(kernel, Xp, t, q, mode="direct", near=False)
    assert 0 < np.count_nonzero(u_far) < len(Xp) or np.count_nonzero(u_far) == len(Xp)
    assert not np.allclose(u_far, u_all)


def _node_ids(kernel, Xp, t, r_of_node, min_level=2):
    """Each node's ID from its full far-field block (rows: all of its far field)."""
    ids = {}
    for b in range(t.n_nodes):
        if t.level[b] < min_level:
            continue
        bg, n = int(t.begin[b]), int(t.count[b])
        far = far_field_mask(Xp, t.centroid[b], t.radius[b], 1.0, bg, bg + n)
        if not far.any():
            continue
        K, _ = o_kernels.kernel_block(kernel, Xp[far], Xp[bg:bg + n])
        ref = o_interp.interpolative_decomposition(K, r_of_node(n))
        ids[b] = (ref["skel_perm"], ref["T"], ref["rank"])
    return ids


def test_tree_full_rank_representation_is_exact():
    kernel = o_kernels.Kernel(o_kernels.GAUSSIAN, h=0.8)
    Xp, t = _small_tree(seed=7, N=900, leaf=40)
    ids = _node_ids(kernel, Xp, t, lambda n: n)
    q = np.random.default_rng(8).standard_normal(len(Xp))
    u_s = o_apply.tree_potential(kernel, Xp, t, q, ids, mode="skeleton")
    u_d = o_apply.tree_potential(kernel, Xp, t, q, mode="direct")
    assert np.max(np.abs(u_s - u_d)) <= 1e-11 * np.max(np.abs(u_d))


@pytest.mark.parametrize("kernel", _KERNELS[:2], ids=["gaussian", "laplace"])
def test_tree_representation_error_is_the_residual_on_the_interaction_lists(kernel):
    """u_skeleton - u_direct at each target = sum over its interaction-list nodes b of
    ((K_b(:, J) P_b - K_b) q_b)(target), with K_b the node's far-field block."""
    Xp, t = _small_tree(seed=9, N=1200, d=3, leaf=40)
    ids = _node_ids(kernel, Xp, t, lambda n: min(n, 6))
    q = np.random.default_rng(10).standard_normal(len(Xp))
    u_s = o_apply.tree_potential(kernel, Xp, t, q, ids, mode="skeleton", near=False)
    u_d = o_apply.tree_potential(kernel, Xp, t, q, mode="direct", near=False)
    far, covered = o_apply.interaction_masks(Xp, t)
    want = np.zeros(len(Xp))
    for b, (skel, T, r) in ids.items():
        bg, n = int(t.begin[b]), int(t.count[b])
        il = far[b] & ~covered[b]
        if not il.any():
            continue
        Kb = o_apply.kernel_values(kernel, Xp[il], Xp[bg:bg + n])
        P = o_interp.assemble_P(skel, T, n)
        want[il] += (Kb[:, skel[:r]] @ P - Kb) @ q[bg:bg + n]
    scale = np.max(np.abs(u_d))
    assert np.max(np.abs((u_s - u_d) - want)) <= 1e-11 * scale
    assert np.max(np.abs(want)) > 1e-8 * scale          # the rank-6 representation is not exact


def test_tree_potential_at_a_target_subset_is_the_same_evaluation():
    kernel = o_kernels.Kernel(o_kernels.GAUSSIAN, h=0.8)
    Xp, t = _small_tree(seed=11, N=1000, leaf=40)
    q = np.random.default_rng(12).standard_normal(len(Xp))
    sub = np.sort(np.random.default_rng(13).choice(len(Xp), 97, replace=False))
    u_all = o_apply.tree_potential(kernel, Xp, t, q, mode="direct")
    u_sub = o_apply.tree_potential(kernel, Xp, t, q, mode="direct", targets=sub)
    assert np.max(np.abs(u_sub - u_all[sub])) <= 1e-13 * np.max(np.abs(u_all))
