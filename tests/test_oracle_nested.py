"""Pins of nested skeletonization (oracle/compress.compress_tree_nested, oracle/apply.nested_*):
the upward pass whose node IDs take their children's skeletons as columns.

* Leaves are the plain per-node compression.
* A parent's columns are exactly its children's skeleton points, in order.
* A kernel of exact rank (the cubic polynomial in d = 3: C(6, 3) = 20) is represented exactly at
  every level, so the nested evaluation reproduces the direct far-field potential to rounding.
* Nested charges compose: with IDs that keep every column (rank = number of columns) the nested
  evaluation equals the direct far-field evaluation.
"""
import numpy as np

import workloads
from oracle import apply as o_apply
from oracle import compress as o_compress
from oracle import kernels as o_kernels
from oracle import tree as o_tree


def _tree(N=2000, d=3, leaf=64, seed=4):
    P = workloads.gaussian_mixture(N=N, d=d, k=3, seed=seed)
    t = o_tree.build_tree(P, leaf)
    return P[t.perm], t


def test_leaves_are_the_plain_compression_and_parents_take_their_childrens_skeletons():
    Xp, t = _tree()
    k = o_kernels.Kernel(o_kernels.GAUSSIAN, h=1.0)
    res = o_compress.compress_tree_nested(Xp, t, k, 1e-6, s0=32, s_max=256)
    for b, r in res.items():
        if t.level[b] == t.depth:
            plain = o_compress.compress_node(Xp, t, b, k, 1e-6, 0, 32, 256)
            assert r.rank == plain.rank and np.array_equal(r.skel_perm, plain.skel_perm)
            assert np.array_equal(r.cols, np.arange(t.count[b]))
        else:
            want = []
            for ch in (2 * b + 1, 2 * b + 2):
                rc = res[ch]
                want.append(rc.cols[rc.skel_perm[:rc.rank]] + t.begin[ch] - t.begin[b])
            assert np.array_equal(r.cols, np.concatenate(want))
            assert r.rank <= r.cols.size and np.all(r.cols < t.count[b])


def test_exact_rank_kernel_is_represented_exactly_at_every_level():
    Xp, t = _tree(N=1500, d=3, leaf=48, seed=6)
    k = o_kernels.Kernel(o_kernels.POLYNOMIAL, h=3.0, c=1.0, p=3)
    res = o_compress.compress_tree_nested(Xp, t, k, 1e-12, s0=64, s_max=256)
    assert all(r.rank <= 20 for r in res.values())
    q = np.random.default_rng(7).standard_normal(len(Xp))
    u_n = o_apply.nested_tree_potential(k, Xp, t, q, res, near=False)
    u_d = o_apply.tree_potential(k, Xp, t, q, mode="direct", near=False)
    assert np.max(np.abs(u_n - u_d)) <= 1e-9 * np.max(np.abs(u_d))


def test_full_rank_nested_charges_compose_to_the_direct_potential():
    Xp, t = _tree(N=800, d=3, leaf=32, seed=8)
    k = o_kernels.Kernel(o_kernels.GAUSSIAN, h=0.7)
    # tol 0 (fixed rank) with s >= columns keeps every column: P is a permutation
    res = {}
    for level in range(t.depth, 1, -1):
        for b in range(t.n_nodes):
            if t.level[b] != level:
                continue
            cols = o_compress.nested_columns(t, b, res)
            r = o_compress.compress_node(Xp, t, b, k, 1e-300, 0, 512, 512, cols=cols)
            r.cols = cols
            res[b] = r
    assert all(r.rank == r.cols.size or r.s < r.cols.size for r in res.values())
    q = np.random.default_rng(9).standard_normal(len(Xp))
    u_n = o_apply.nested_tree_potential(k, Xp, t, q, res)
    u_d = o_apply.tree_potential(k, Xp, t, q, mode="direct")
    full = all(r.rank == r.cols.size for r in res.values())
    if full:
        assert np.max(np.abs(u_n - u_d)) <= 1e-10 * np.max(np.abs(u_d))
    else:                               # a far field smaller than the columns caps the rank
        assert np.linalg.norm(u_n - u_d) <= 1e-2 * np.linalg.norm(u_d)
