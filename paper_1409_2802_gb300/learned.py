"""Training of the learned row proposal on exact leverage scores, on the GPU.

Argument marshalling and bookkeeping only: every arithmetic step is a libffc
call (see ``ffc``). The targets are the statistical leverage scores of §3
(Def. "Statistical Leverage"), the row distribution that the paper finds
best (§4.1.3 "Leverage sampling") but that needs the full block.

For a training node (centroid x_c, radius rho, positions [b, b + n) of the
points in tree order):

* far field T = {y outside the node : ||y - x_c|| >= xi rho} (§4.1 steps 2-3),
  ``ffc_far_field``;
* K = K(T, node sources) in FP64 (``ffc_eval_block``);
* targets l_i = leverage of row i of K at its eps-rank (``ffc_leverage``),
  normalised per node inside the loss;
* features of every far-field row (``ffc_features``).

Training: Adam (``ffc_adam_step``) on the mean per-node softmax cross-entropy
(``ffc_mlp_loss_grad``), one step per batch of whole nodes, batches visited in
a seeded order each epoch.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np
import torch

from . import ffc


@dataclass
class TrainingSet:
    feats: torch.Tensor                  # R x 12 float32 (CUDA)
    targets: torch.Tensor                # R float64 leverage scores (CUDA)
    node_rows: list                      # rows per node, in storage order
    ranks: list                          # eps-rank of each node's block
    batches: list = field(default_factory=list)   # (row_begin, row_end, node_off CUDA int64)

    @property
    def n_nodes(self) -> int:
        return len(self.node_rows)


def node_block(points_perm, tree: ffc.DeviceTree, node: int, kernel: ffc.Kernel, proj, xi=1.0):
    """(far-field block K as (n, m) storage, features m x 12) of one node, or None."""
    b = int(tree.begin[node].item())
    n = int(tree.count[node].item())
    x_c = tree.centroid[node].contiguous()
    rho = float(tree.radius[node].item())
    far = ffc.ffc_far_field(points_perm, x_c, rho, xi, b, b + n)
    m = far.numel()
    if m == 0:
        return None
    K = torch.empty((n, m), dtype=torch.float64, device=points_perm.device)
    ffc.ffc_eval_block(kernel, points_perm, far, points_perm[b:b + n], precision=ffc.FP64, K=K)
    F = ffc.ffc_features(kernel, points_perm, far, x_c, rho, proj)
    return K, F


def build_training_set(sources, eps=1e-6, batch_nodes=8, seed=0, xi=1.0, block_bytes=24 << 30) -> TrainingSet:
    """``sources``: iterable of (points_perm, tree, nodes, kernel, proj) tuples.

    The leverage targets of up to ``block_bytes`` of far-field blocks are
    computed in one batched call. Nodes are stored in a seeded random order
    and grouped into training batches of ``batch_nodes`` consecutive nodes.
    """
    parts = []
    pending, held = [], 0

    def flush():
        nonlocal pending, held
        if not pending:
            return
        outs, _ = ffc.ffc_leverage_batched([K for K, _ in pending], eps)
        for (K, F), (lev, _, r) in zip(pending, outs):
            if r > 0:
                parts.append((F, lev, r))
        pending, held = [], 0

    for points_perm, tree, nodes, kernel, proj in sources:
        for node in nodes:
            out = node_block(points_perm, tree, int(node), kernel, proj, xi)
            if out is None:
                continue
            nbytes = out[0].numel() * 8
            if pending and held + nbytes > block_bytes:
                flush()
            pending.append(out)
            held += nbytes
    flush()
    if not parts:
        raise ValueError("no training node has a far field")
    order = np.random.Generator(np.random.PCG64(seed)).permutation(len(parts))
    parts = [parts[i] for i in order]
    feats = torch.cat([p[0] for p in parts], dim=0).contiguous()
    targets = torch.cat([p[1] for p in parts], dim=0).contiguous()
    rows = [int(p[0].shape[0]) for p in parts]
    ts = TrainingSet(feats, targets, rows, [int(p[2]) for p in parts])
    start = np.concatenate([[0], np.cumsum(rows)])
    dev = feats.device
    for a in range(0, len(parts), batch_nodes):
        e = min(a + batch_nodes, len(parts))
        off = torch.tensor(start[a:e + 1] - start[a], dtype=torch.int64, device=dev)
        ts.batches.append((int(start[a]), int(start[e]), off))
    return ts


def mean_loss(ts: TrainingSet, params) -> float:
    """Mean over nodes of the cross-entropy of ``params`` on the whole set."""
    tot = 0.0
    for r0, r1, off in ts.batches:
        loss, _ = ffc.ffc_mlp_loss_grad(params, ts.feats[r0:r1], ts.targets[r0:r1], off)
        tot += loss * (off.numel() - 1)
    return tot / ts.n_nodes


def train(ts: TrainingSet, params0, epochs=20, lr=1e-3, seed=0, beta1=0.9, beta2=0.999, eps=1e-8):
    """Adam on the batches of ``ts``; returns (params float32 CUDA, per-step losses)."""
    dev = ts.feats.device
    params = torch.as_tensor(np.asarray(params0, dtype=np.float32)).to(dev).contiguous()
    m = torch.zeros_like(params)
    v = torch.zeros_like(params)
    grad = torch.empty_like(params)
    rng = np.random.Generator(np.random.PCG64(seed))
    losses = []
    step = 0
    for _ in range(epochs):
        for bi in rng.permutation(len(ts.batches)):
            r0, r1, off = ts.batches[bi]
            loss, _ = ffc.ffc_mlp_loss_grad(params, ts.feats[r0:r1], ts.targets[r0:r1], off, grad=grad)
            step += 1
            ffc.ffc_adam_step(params, grad, m, v, step, lr, beta1, beta2, eps)
            losses.append(loss)
    return params, losses
