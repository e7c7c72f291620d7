"""PCA median-split binary tree and per-node far-field geometry (oracle side).

Test infrastructure (see ``oracle/__init__``).

The paper only names a space-partitioning tree (§2: a kd-tree or octree
groups the sources so that far fields can be identified) and the node
geometry of its setup (§4.1: centre x_c, radius rho = largest distance from
x_c to a source). The tree used by the workloads is defined here:

* depth D = smallest D with ceil(N / 2^D) <= leaf_size; a complete binary
  tree in heap order (node 0 is the root, the children of i are 2i+1, 2i+2;
  level l holds nodes 2^l - 1 .. 2^(l+1) - 2);
* a node holds positions [begin, begin + count) of the permutation ``perm``;
  its left child takes the first floor(count/2) positions;
* x_c = mean of the node's points, rho = max ||x - x_c|| over them;
* split direction = principal direction of the node's centred points from 32
  power iterations v <- C^T (C v) / ||C^T (C v)|| starting at (1,...,1)/sqrt(d),
  with the sign chosen so that the largest-magnitude component (lowest index
  on ties) is positive;
* the node's points are ordered by (projection onto v, original index) and
  the lower half goes left.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

POWER_ITERS = 32


def tree_depth(N: int, leaf_size: int) -> int:
    D = 0
    while -(-N // (1 << D)) > leaf_size:
        D += 1
    return D


@dataclass
class Tree:
    depth: int
    perm: np.ndarray        # int64[N]: position -> original point index
    begin: np.ndarray       # int64[n_nodes]
    count: np.ndarray       # int64[n_nodes]
    level: np.ndarray       # int32[n_nodes]
    centroid: np.ndarray    # float64[n_nodes, d]
    radius: np.ndarray      # float64[n_nodes]

    @property
    def n_nodes(self) -> int:
        return int(self.begin.shape[0])

    def level_nodes(self, level: int) -> range:
        return range((1 << level) - 1, (1 << (level + 1)) - 1)


def principal_direction(C: np.ndarray) -> np.ndarray:
    d = C.shape[1]
    v = np.full(d, 1.0 / np.sqrt(d))
    for _ in range(POWER_ITERS):
        w = C.T @ (C @ v)
        nrm = float(np.sqrt(np.sum(w * w)))
        if nrm == 0.0:
            break
        v = w / nrm
    i = int(np.argmax(np.abs(v)))
    if v[i] < 0.0:
        v = -v
    return v


def node_layout(N: int, depth: int):
    """begin/count/level of every node; they depend only on N and the depth."""
    n_nodes = (1 << (depth + 1)) - 1
    begin = np.zeros(n_nodes, dtype=np.int64)
    count = np.zeros(n_nodes, dtype=np.int64)
    level = np.zeros(n_nodes, dtype=np.int32)
    count[0] = N
    for i in range(n_nodes):
        if 2 * i + 2 < n_nodes:
            left = count[i] // 2
            begin[2 * i + 1], count[2 * i + 1] = begin[i], left
            begin[2 * i + 2], count[2 * i + 2] = begin[i] + left, count[i] - left
            level[2 * i + 1] = level[2 * i + 2] = level[i] + 1
    return begin, count, level


def build_tree(points, leaf_size: int) -> Tree:
    X = np.asarray(points, dtype=np.float64)
    N, d = X.shape
    D = tree_depth(N, leaf_size)
    begin, count, level = node_layout(N, D)
    n_nodes = begin.shape[0]
    perm = np.arange(N, dtype=np.int64)
    centroid = np.zeros((n_nodes, d))
    radius = np.zeros(n_nodes)
    for i in range(n_nodes):
        b, c = int(begin[i]), int(count[i])
        idx = perm[b:b + c].copy()
        P = X[idx]
        xc = P.mean(axis=0)
        C = P - xc
        centroid[i] = xc
        radius[i] = float(np.sqrt(np.max(np.sum(C * C, axis=1)))) if c > 0 else 0.0
        if level[i] < D:
            v = principal_direction(C)
            proj = C @ v
            order = np.lexsort((idx, proj))
            perm[b:b + c] = idx[order]
    return Tree(D, perm, begin, count, level, centroid, radius)
