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


# ---------------------------------------------------------------------------
# the standard training recipe: leaf nodes of the d = 128 and d = 1000 generators

def recipe_sources(seed: int = 0, nodes_d128: int = 100, nodes_d1000: int = 100, device="cuda"):
    """(points_perm, tree, nodes, kernel, proj) of the two training generators.

    d = 128: N = 262,144 points of the decaying 16-component mixture, leaf 256,
    Laplace kernel; d = 1000: N = 100,000 points of intrinsic dimension 10,
    leaf 512, Gaussian kernel with h = the median pairwise distance. Nodes are
    a seeded choice among the leaves.
    """
    import workloads
    out = []
    specs = (
        (workloads.decaying_mixture(262144, 128, 16, seed=seed), 256, None, nodes_d128),
        (workloads.low_intrinsic(100000, 10, 1000, seed=seed), 512, "median", nodes_d1000),
    )
    for X, leaf, h, count in specs:
        kernel = (ffc.Kernel(ffc.LAPLACE) if h is None
                  else ffc.Kernel(ffc.GAUSSIAN, h=workloads.median_pairwise_distance(X)))
        Xd = torch.as_tensor(X).to(device)
        tree = ffc.ffc_build_tree(Xd, leaf)
        Xp = Xd[tree.perm].contiguous()
        first = (1 << tree.depth) - 1
        leaves = np.arange(first, tree.n_nodes)
        pick = np.random.Generator(np.random.PCG64(seed + leaf)).choice(leaves, size=min(count, leaves.size),
                                                                        replace=False)
        proj = torch.as_tensor(workloads.projections(X.shape[1], seed=seed + 7)).to(device)
        out.append((Xp, tree, sorted(int(i) for i in pick), kernel, proj))
    return out


def train_standard(seed: int = 0, epochs: int = 30, lr: float = 2e-3, nodes_per_generator: int = 100,
                   device="cuda"):
    """Train the proposal with the standard recipe; returns (params, info dict)."""
    import time

    import workloads
    t0 = time.perf_counter()
    ts = build_training_set(recipe_sources(seed, nodes_per_generator, nodes_per_generator, device), eps=1e-6,
                            batch_nodes=8, seed=seed)
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    theta0 = workloads.mlp_init(seed + 1)
    loss0 = mean_loss(ts, torch.as_tensor(theta0).to(device))
    params, losses = train(ts, theta0, epochs=epochs, lr=lr, seed=seed)
    loss1 = mean_loss(ts, params)
    torch.cuda.synchronize()
    t2 = time.perf_counter()
    info = {"nodes": ts.n_nodes, "rows": int(ts.feats.shape[0]), "targets_s": round(t1 - t0, 1),
            "train_s": round(t2 - t1, 1), "adam_steps": len(losses), "loss_start": round(loss0, 4),
            "loss_end": round(loss1, 4), "epochs": epochs, "lr": lr}
    del ts
    return params, info
