"""The outgoing representation from an ID (oracle side).

Test infrastructure (see ``oracle/__init__``).

§2.1.3, after the ID's error theorem: with K ~ C P, C = K(:, J) the skeleton
columns and P (r x n) containing I_r, a node's source charges q (n) become
equivalent skeleton charges q~ = P q (r), and the potential its sources
induce at a target y_i is u_i = (K q)_i ~ (C q~)_i = sum_j K(y_i, x~_j) q~_j,
x~_j the skeleton points. The charges take O(n r) work, each potential O(r)
kernel evaluations. ``tree_potential`` uses the representations of every
node of a tree to evaluate the potential at every point (the treecode the
representation exists for; see the comment above it).

With the shared output convention (``interp``), P = [I_r T] Pi^T, so
q~ = q[skel_perm[:r]] + T q[skel_perm[r:]].
"""
from __future__ import annotations

import numpy as np

from .kernels import Kernel, kernel_block


def skeleton_charges(skel_perm, T, q):
    """q~ = P q for P = [I_r T] Pi^T: the skeleton's own charges plus T times the others'."""
    skel_perm = np.asarray(skel_perm, dtype=np.int64)
    T = np.asarray(T, dtype=np.float64)
    q = np.asarray(q, dtype=np.float64)
    r = T.shape[0]
    return q[skel_perm[:r]] + T @ q[skel_perm[r:]]


def direct_potential(kernel: Kernel, Y, X, q):
    """u = K q at the targets Y for sources X with charges q (the sum the representation replaces)."""
    K, log_scale = kernel_block(kernel, Y, X)
    return K @ np.asarray(q, dtype=np.float64), log_scale


def id_potential(kernel: Kernel, Y, X, skel_perm, r, q_tilde):
    """u~ = C q~ = sum_j K(y, x~_j) q~_j over the r skeleton points x~_j = X[skel_perm[j]].

    C is taken from the block of all sources, so that it carries the same scale as
    ``direct_potential``'s (the Laplace block is scaled by its largest entry)."""
    K, log_scale = kernel_block(kernel, Y, X)
    C = K[:, np.asarray(skel_perm, dtype=np.int64)[:r]]
    return C @ np.asarray(q_tilde, dtype=np.float64), log_scale


# ---------------------------------------------------------------------------
# The representation over a tree: a treecode evaluation with the paper's
# far-field test as the admissibility rule.
#
# Every node b at level >= min_level has a far field far(b) = the points
# outside b at distance >= xi rho_b from its centroid (§4.1 setup, per node).
# A target y takes b's outgoing representation when y is in far(b) and in the
# far field of none of b's ancestors at level >= min_level (the topmost far
# node on each path from a level-min_level node down to a leaf: "b is in y's
# interaction list"); a leaf reached without any far node on its path is y's
# near field and is summed directly, without y's own point. Every source other
# than y is then counted exactly once:
#     u(y) = sum_{b in IL(y)} sum_j K(y, x~_j) q~_j + sum_{x in near(y), x != y} K(y, x) q(x)
# with q~ = P_b q_b, x~ the skeleton points of b. Replacing the skeleton sum by
# sum_{x in b} K(y, x) q(x) (mode "direct") gives the exact far-field value
# the representation approximates. Potentials are returned multiplied by
# exp(-log_scale) (a common scale for the Laplace kernel's range).


def kernel_values(kernel: Kernel, Y, X, log_scale=0.0):
    """K(Y, X) exp(-log_scale) from the paper's formulas (the Laplace power through logarithms).

    Coincident points give an infinite Laplace value; callers exclude them."""
    from .kernels import GAUSSIAN, LAPLACE, POLYNOMIAL, squared_distances
    Y = np.asarray(Y, dtype=np.float64)
    X = np.asarray(X, dtype=np.float64)
    if kernel.kind == GAUSSIAN:
        return np.exp(-squared_distances(Y, X) / (2.0 * kernel.h * kernel.h) - log_scale)
    if kernel.kind == LAPLACE:
        d = Y.shape[1]
        with np.errstate(divide="ignore"):
            return np.exp(-0.5 * (d - 2) * np.log(squared_distances(Y, X)) - log_scale)
    if kernel.kind == POLYNOMIAL:
        return (Y @ X.T / kernel.h + kernel.c) ** kernel.p * np.exp(-log_scale)
    raise ValueError(kernel.kind)


def interaction_masks(Xp, tree, xi=1.0, min_level=2, targets=None):
    """(far, covered): per node b at level >= min_level, far[b] marks the targets in b's far field and
    covered[b] those in the far field of an ancestor at level >= min_level; b is in y's interaction list
    where far[b] & ~covered[b]. Targets: the points at positions ``targets`` (default: all, tree order)."""
    Xp = np.asarray(Xp, dtype=np.float64)
    pos = np.arange(len(Xp)) if targets is None else np.asarray(targets, dtype=np.int64)
    Y = Xp[pos]
    far, covered = {}, {}
    for b in range(tree.n_nodes):
        if tree.level[b] < min_level:
            continue
        bg, n = int(tree.begin[b]), int(tree.count[b])
        diff = Y - np.asarray(tree.centroid[b], dtype=np.float64)[None, :]
        thr = float(xi) * float(tree.radius[b])
        far[b] = (np.sum(diff * diff, axis=1) >= thr * thr) & ~((pos >= bg) & (pos < bg + n))
        p = (b - 1) // 2
        covered[b] = (covered[p] | far[p]) if b > 0 and tree.level[p] >= min_level else np.zeros(pos.size, bool)
    return far, covered


def tree_potential(kernel: Kernel, Xp, tree, q, ids=None, xi=1.0, min_level=2, mode="skeleton", near=True,
                   log_scale=0.0, targets=None):
    """u at the points at positions ``targets`` (default: every point, tree order) for charges q (tree
    order); ids: node -> (skel_perm, T, r) of the node's ID (mode "skeleton"; a node without one is summed
    directly), ignored in mode "direct"."""
    Xp = np.asarray(Xp, dtype=np.float64)
    q = np.asarray(q, dtype=np.float64)
    pos = np.arange(len(Xp)) if targets is None else np.asarray(targets, dtype=np.int64)
    u = np.zeros(pos.size)
    far, covered = interaction_masks(Xp, tree, xi, min_level, pos)
    for b in far:
        bg, n = int(tree.begin[b]), int(tree.count[b])
        sel = np.flatnonzero(far[b] & ~covered[b])
        if sel.size == 0:
            continue
        Xb, qb = Xp[bg:bg + n], q[bg:bg + n]
        if mode == "skeleton" and ids is not None and ids.get(b) is not None:
            skel, T, r = ids[b]
            u[sel] += kernel_values(kernel, Xp[pos[sel]], Xb[np.asarray(skel)[:r]], log_scale) @ \
                skeleton_charges(skel, T, qb)
        else:
            u[sel] += kernel_values(kernel, Xp[pos[sel]], Xb, log_scale) @ qb
    if near:
        for b in far:
            if tree.level[b] != tree.depth:
                continue
            bg, n = int(tree.begin[b]), int(tree.count[b])
            sel = np.flatnonzero(~far[b] & ~covered[b])
            if sel.size == 0:
                continue
            Kb = kernel_values(kernel, Xp[pos[sel]], Xp[bg:bg + n], log_scale)
            own = (pos[sel][:, None] == np.arange(bg, bg + n)[None, :])
            Kb[own] = 0.0                                   # without the target's own point
            u[sel] += Kb @ q[bg:bg + n]
    return u


def direct_sum_without_self(kernel: Kernel, Xp, q, log_scale=0.0):
    """u_i = sum_{j != i} K(x_i, x_j) q_j over all points: the sum a tree evaluation reorganises."""
    K = kernel_values(kernel, Xp, Xp, log_scale)
    np.fill_diagonal(K, 0.0)
    return K @ np.asarray(q, dtype=np.float64)


def nested_skeleton_charges(tree, results: dict, q, min_level=2):
    """Skeleton charges of every node of a nested compression (compress.compress_tree_nested), from the
    leaves up: q~_b = P_b q_cols with q_cols the leaf's charges, or the children's skeleton charges
    (a child without a usable ID contributes its points' charges)."""
    from .compress import usable
    q = np.asarray(q, dtype=np.float64)
    qt = {}
    for level in range(tree.depth, min_level - 1, -1):
        for b in range(tree.n_nodes):
            if tree.level[b] != level:
                continue
            bg, n = int(tree.begin[b]), int(tree.count[b])
            if level == tree.depth:
                qc = q[bg:bg + n]
            else:
                parts = []
                for ch in (2 * b + 1, 2 * b + 2):
                    cb, cn = int(tree.begin[ch]), int(tree.count[ch])
                    parts.append(qt[ch] if usable(results[ch]) else q[cb:cb + cn])
                qc = np.concatenate(parts)
            r = results[b]
            qt[b] = skeleton_charges(r.skel_perm, r.T, qc) if usable(r) else None
    return qt


def nested_tree_potential(kernel: Kernel, Xp, tree, q, results: dict, xi=1.0, min_level=2, near=True,
                          log_scale=0.0, targets=None):
    """tree_potential with the nested representations: node b's skeleton points are its points
    cols_b[skel_b[0:r_b]] and its charges come from nested_skeleton_charges."""
    from .compress import usable
    qt = nested_skeleton_charges(tree, results, q, min_level)
    ids = {}
    for b, r in results.items():
        if usable(r):
            ids[b] = (r.cols[r.skel_perm], r.T, r.rank, qt[b])
    Xp = np.asarray(Xp, dtype=np.float64)
    q = np.asarray(q, dtype=np.float64)
    pos = np.arange(len(Xp)) if targets is None else np.asarray(targets, dtype=np.int64)
    u = np.zeros(pos.size)
    far, covered = interaction_masks(Xp, tree, xi, min_level, pos)
    for b in far:
        bg, n = int(tree.begin[b]), int(tree.count[b])
        sel = np.flatnonzero(far[b] & ~covered[b])
        if sel.size == 0:
            continue
        if b in ids:
            pts, _, r, qtb = ids[b]
            u[sel] += kernel_values(kernel, Xp[pos[sel]], Xp[bg + pts[:r]], log_scale) @ qtb
        else:
            u[sel] += kernel_values(kernel, Xp[pos[sel]], Xp[bg:bg + n], log_scale) @ q[bg:bg + n]
    if near:
        for b in far:
            if tree.level[b] != tree.depth:
                continue
            bg, n = int(tree.begin[b]), int(tree.count[b])
            sel = np.flatnonzero(~far[b] & ~covered[b])
            if sel.size == 0:
                continue
            Kb = kernel_values(kernel, Xp[pos[sel]], Xp[bg:bg + n], log_scale)
            Kb[pos[sel][:, None] == np.arange(bg, bg + n)[None, :]] = 0.0
            u[sel] += Kb @ q[bg:bg + n]
    return u
