"""Per-node sampled-row ID over a tree (oracle side).

Test infrastructure (see ``oracle/__init__``).

For every node at level >= 2 (each node's own far field, §4.1 steps 2-3 with
x_c = the node centroid and xi = 1): sample s far-field rows uniformly
(§2.2), evaluate K'(rows, node sources), compute its ID at relative
tolerance tol (§2.1.3, App. A.1).

Reading of "s = 2 x rank" (the rank is only known after the QR): start at
s = s0 and run the pivoted QR in tolerance mode for at most s/2 steps; if the
tolerance is not met, double s and start again. The sampler is prefix
consistent, so the first s rows are kept. When the sample already holds the
whole far field (the sampler returned fewer than s rows) the QR may run to
min(s, n) steps; the rank never exceeds
r_cap = s_max / 2. A node that cannot meet the tolerance within those limits
keeps its last ID with status TOL_NOT_REACHED.

With a learned ``Proposal`` the s rows of each attempt come from
``proposal.propose_from_mask`` (network weights over the candidate pool,
weighted draw without replacement) instead of the uniform sampler; its keys
do not depend on s, so a larger attempt extends the smaller one as well.
With ``ranked_rows`` the rows of each attempt are the first s of that list
instead (a draw made elsewhere and checked on its own, passed in like any
other random input); everything after the draw is the same.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

from .interp import interpolative_decomposition
from .kernels import Kernel, kernel_block
from .proposal import propose_from_mask
from .sampling import far_field_mask, sample_uniform_from_mask

STATUS_OK = 0
STATUS_FARFIELD_EMPTY = 5
STATUS_TOL_NOT_REACHED = 7


@dataclass
class NodeResult:
    node: int
    s: int                  # rows actually sampled
    rows: np.ndarray        # sampled positions (tree order)
    rank: int
    skel_perm: np.ndarray   # node-local column indices
    T: np.ndarray
    r22_rel: float
    log_scale: float
    far_count: int
    status: int
    attempts: list = field(default_factory=list)   # s values tried
    cols: np.ndarray | None = None                   # nested form: node-local points of the ID's columns


@dataclass
class Proposal:
    theta32: np.ndarray     # FP32 master parameters of the proposal network
    proj: np.ndarray        # 8 x d random directions of the projection features
    pool_rows: int = 0      # 0: the whole far field; else a uniform pool of this size


def rank_cap(s_eff: int, n: int, all_rows: bool, r_cap: int) -> int:
    return min(n, r_cap, s_eff if all_rows else s_eff // 2)


def compress_node(Xp, tree, node, kernel: Kernel, tol, seed, s0=128, s_max=2048, xi=1.0,
                  proposal: Proposal | None = None, ranked_rows=None, cols=None):
    """The sampled-row ID of one node; ``cols`` (node-local point indices) restricts the ID's columns to
    those points (the nested form), default all of the node's points. skel_perm indexes the columns."""
    b, c = int(tree.begin[node]), int(tree.count[node])
    far = far_field_mask(Xp, tree.centroid[node], tree.radius[node], xi, b, b + c)
    far_count = int(far.sum())
    X_node = Xp[b:b + c]
    if cols is not None:
        X_node = X_node[np.asarray(cols, dtype=np.int64)]
        c = X_node.shape[0]
    r_cap = s_max // 2
    s = s0
    tried = []
    while True:
        tried.append(s)
        if ranked_rows is not None:
            rows = np.asarray(ranked_rows, dtype=np.int64)[:s]
        elif proposal is None:
            rows = sample_uniform_from_mask(far, s, seed, node)
        else:
            rows = propose_from_mask(far, Xp, s, seed, node, tree.centroid[node], tree.radius[node],
                                     kernel, proposal.proj, proposal.theta32, proposal.pool_rows)
        if rows.size == 0:
            return NodeResult(node, 0, rows, 0, np.arange(c), np.zeros((0, c)), 0.0, 0.0,
                              far_count, STATUS_FARFIELD_EMPTY, tried)
        # the whole far field is in the sample exactly when the sampler came
        # back with fewer rows than asked for (|T| < s); when |T| == s the
        # next doubling finds that out
        all_rows = rows.size < s
        K, log_scale = kernel_block(kernel, Xp[rows], X_node)
        cap = rank_cap(rows.size, c, all_rows, r_cap)
        idr = interpolative_decomposition(K, cap, tol)
        done = idr["r22_rel"] <= tol
        if done or all_rows or 2 * s > s_max:
            st = STATUS_OK if done else STATUS_TOL_NOT_REACHED
            return NodeResult(node, int(rows.size), rows, idr["rank"], idr["skel_perm"], idr["T"],
                              idr["r22_rel"], log_scale, far_count, st, tried)
        s *= 2


def compress_tree(Xp, tree, kernel: Kernel, tol, seed=0, min_level=2, s0=128, s_max=2048,
                  nodes=None, proposal: Proposal | None = None):
    """Compress every node at level >= min_level (or just ``nodes``)."""
    if nodes is None:
        nodes = [i for i in range(tree.n_nodes) if tree.level[i] >= min_level]
    return [compress_node(Xp, tree, i, kernel, tol, seed, s0, s_max, proposal=proposal)
            for i in nodes]


# ---------------------------------------------------------------------------
# Nested skeletonization (the upward pass of a treecode built on these IDs, §2
# "outgoing representation of each node by combining the representations of its
# children"; ASKIT, §1): levels are compressed from the leaves up. A leaf's ID
# has the leaf's points as its columns; a node above has its children's skeleton
# points as its columns (left child's, then right child's, each in its pivot
# order), so its skeleton is a subset of theirs and its charges are
# q~ = P [q~_left; q~_right]. A child without a usable ID (status other than OK
# or TOL_NOT_REACHED, or no far field) contributes all of its points. Rows: the
# node's own far-field sample, as in the plain form.

def usable(res: NodeResult) -> bool:
    return res.status in (STATUS_OK, STATUS_TOL_NOT_REACHED) and res.s > 0


def nested_columns(tree, node, results: dict):
    """Node-local point indices of the ID columns of `node` in the nested form."""
    b = int(tree.begin[node])
    if tree.level[node] == tree.depth:
        return np.arange(int(tree.count[node]), dtype=np.int64)
    cols = []
    for ch in (2 * node + 1, 2 * node + 2):
        cb, cn = int(tree.begin[ch]), int(tree.count[ch])
        rc = results[ch]
        if usable(rc):
            own = rc.cols[rc.skel_perm[:rc.rank]]
        else:
            own = np.arange(cn, dtype=np.int64)
        cols.append(own + (cb - b))
    return np.concatenate(cols).astype(np.int64)


def compress_tree_nested(Xp, tree, kernel: Kernel, tol, seed=0, min_level=2, s0=128, s_max=2048):
    """Every node at level >= min_level, from the deepest level up; result.cols holds each node's columns."""
    results = {}
    for level in range(tree.depth, min_level - 1, -1):
        for node in range(tree.n_nodes):
            if tree.level[node] != level:
                continue
            cols = nested_columns(tree, node, results)
            r = compress_node(Xp, tree, node, kernel, tol, seed, s0, s_max, cols=cols)
            r.cols = cols
            results[node] = r
    return results
