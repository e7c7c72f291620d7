"""The outgoing representation from an ID (oracle side).

Test infrastructure (see ``oracle/__init__``).

§2.1.3, after the ID's error theorem: with K ~ C P, C = K(:, J) the skeleton
columns and P (r x n) containing I_r, a node's source charges q (n) become
equivalent skeleton charges q~ = P q (r), and the potential its sources
induce at a target y_i is u_i = (K q)_i ~ (C q~)_i = sum_j K(y_i, x~_j) q~_j,
x~_j the skeleton points. The charges take O(n r) work, each potential O(r)
kernel evaluations.

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
