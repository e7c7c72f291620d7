"""Autotuner of the tree compression's QR launch shape.

The pivoted QR runs as cooperative launches over sub-batches of a round's
sampled blocks (see ``ffc_compress_tree``). Two knobs shape those launches
without changing what is computed (only the FP32 summation order of the
mixed-precision update can differ):

* ``qr_big_min_s``: the smallest sample size whose rounds use the
  register-resident QR variant (2 CTAs per SM, 128 registers: a column of up
  to 2,048 FP32 rows stays in registers across a step). Mixed precision only.
* ``qr_l2_budget_mb``: the bytes of sampled blocks one launch holds. Below L2,
  a launch's steps run from L2; above, more blocks share one launch.

The tuner times whole compression calls on the caller's tree, with CUDA
events on the call's stream after one untimed call per candidate. It is a
coordinate search:
1. the variant threshold at the default budget;
2. the budget at the best threshold.

It returns the fastest setting and the table of everything it timed.

``tune_eval`` picks the evaluation path of the mixed-precision Gaussian and
polynomial blocks: the mma.sync tiles or one of the tcgen05 tile variants
(output tile, coordinates per stage, stage count). The choice is keyed by
(d, precision, kernel, n-bucket, s, point dtype) and cached; it times single
blocks of s rows against n sources of that bucket. ``tune_tree_eval`` times
the candidates where they run: the evaluation phase of a one-round compression
call on the caller's tree.
"""
from __future__ import annotations

import json
import os
import time

import torch

from . import ffc

BIG_MIN_S = (512, 1024, 2048, 1 << 30)   # 1 << 30: never
L2_BUDGET_MB = (64, 96, 128)


def _time_call(points_perm, tree, kernel, stream, reps, **kw) -> float:
    res = ffc.ffc_compress_tree(points_perm, tree, kernel, stream=stream, **kw)   # untimed
    times = []
    for _ in range(reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        res = ffc.ffc_compress_tree(points_perm, tree, kernel, stream=stream, result=res, **kw)
        e1.record(stream)
        e1.synchronize()
        times.append(e0.elapsed_time(e1))
    res.close()
    return min(times)


def tune_tree(points_perm, tree: ffc.DeviceTree, kernel: ffc.Kernel, precision=ffc.MIXED, reps: int = 1,
              stream=None, **compress_kw) -> dict:
    """Fastest (qr_big_min_s, qr_l2_budget_mb) for this tree; ``compress_kw`` are the other
    arguments of ``ffc_compress_tree`` (tol, s0, s_max, proposal, ...), fixed during the search."""
    t0 = time.perf_counter()
    stream = stream if stream is not None else torch.cuda.current_stream()
    table = []

    def run(big, budget):
        # a candidate the device cannot run (e.g. out of memory) is skipped, not fatal
        try:
            ms = _time_call(points_perm, tree, kernel, stream, reps, precision=precision, qr_big_min_s=big,
                            qr_l2_budget_mb=budget, **compress_kw)
        except ffc.FFCError as e:
            table.append({"qr_big_min_s": big, "qr_l2_budget_mb": budget, "error": str(e)[:120]})
            return float("inf")
        table.append({"qr_big_min_s": big, "qr_l2_budget_mb": budget, "ms": round(ms, 3)})
        return ms

    default_budget = 96
    if precision == ffc.MIXED:
        bigs = {b: run(b, default_budget) for b in BIG_MIN_S}
        big = min(bigs, key=bigs.get)
    else:
        big = BIG_MIN_S[-1]            # the register-resident variant is FP32 only
        bigs = {big: run(big, default_budget)}
    budgets = {default_budget: bigs[big]}
    for b in L2_BUDGET_MB:
        if b not in budgets:
            budgets[b] = run(big, b)
    budget = min(budgets, key=budgets.get)
    if budgets[budget] == float("inf"):
        raise ffc.FFCError(ffc.FFC_E_CUDA, "autotune: no candidate launch shape ran")
    return {"qr_big_min_s": big, "qr_l2_budget_mb": budget, "ms": round(budgets[budget], 3), "table": table,
            "seconds": round(time.perf_counter() - t0, 1)}


EVAL_CANDIDATES = (ffc.EVAL_MMA_SYNC,) + tuple(ffc.EVAL_TCGEN05_TILE0 + v for v in range(ffc.EVAL_TCGEN05_TILES))
N_BUCKETS = (256, 1024, 4096, 16384, 65536)
_EVAL_CACHE: dict = {}


def n_bucket(n: int) -> int:
    """The smallest bucket at or above n (the largest bucket beyond it)."""
    for b in N_BUCKETS:
        if n <= b:
            return b
    return N_BUCKETS[-1]


def _eval_key(d, precision, kind, nb, s, dtype):
    return f"d={d},precision={precision},kernel={kind},n={nb},s={s},dtype={str(dtype).split('.')[-1]}"


def tune_eval(kernel: ffc.Kernel, d: int, n: int, precision=ffc.MIXED, s: int = 2048, dtype=torch.float64,
              reps: int = 3, cache_path: str | None = None, device=None) -> dict:
    """Fastest evaluation path for one s x n block in d dimensions (synthetic standard-normal points of the
    given dtype; the time does not depend on the values). Only the mixed-precision Gaussian and polynomial
    blocks have a choice; the others return EVAL_DEFAULT. Results are cached in memory and, with
    ``cache_path``, in a JSON file."""
    if precision != ffc.MIXED or kernel.kind == ffc.LAPLACE:
        return {"eval_path": ffc.EVAL_DEFAULT, "source": "no choice"}
    nb = n_bucket(n)
    key = _eval_key(d, precision, kernel.kind, nb, s, dtype)
    if key not in _EVAL_CACHE and cache_path and os.path.exists(cache_path):
        with open(cache_path) as f:
            _EVAL_CACHE.update(json.load(f))
    if key in _EVAL_CACHE:
        return dict(_EVAL_CACHE[key], source="cache")
    dev = device if device is not None else torch.device("cuda", torch.cuda.current_device())
    g = torch.Generator(device=dev).manual_seed(d * 7919 + nb)
    X = torch.randn(nb, d, device=dev, dtype=dtype, generator=g)
    Y = torch.randn(2 * s, d, device=dev, dtype=dtype, generator=g)
    rows = torch.arange(s, dtype=torch.int64, device=dev)
    ctr = X.double().mean(0)
    K = torch.empty((nb, s), dtype=torch.float32, device=dev)
    table = {}
    try:
        for path in EVAL_CANDIDATES:
            ffc.ffc_set_eval_path(path)
            ffc.ffc_eval_block(kernel, Y, rows, X, precision=precision, center=ctr, K=K)   # untimed
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record()
            for _ in range(reps):
                ffc.ffc_eval_block(kernel, Y, rows, X, precision=precision, center=ctr, K=K)
            e1.record()
            e1.synchronize()
            table[path] = e0.elapsed_time(e1) / reps
    finally:
        ffc.ffc_set_eval_path(ffc.EVAL_DEFAULT)
    best = min(table, key=table.get)
    out = {"eval_path": best, "ms": round(table[best], 4), "table": {str(k): round(v, 4) for k, v in table.items()}}
    _EVAL_CACHE[key] = out
    if cache_path:
        with open(cache_path, "w") as f:
            json.dump(_EVAL_CACHE, f, indent=1, sort_keys=True)
    return dict(out, source="measured")


def tune_tree_eval(points_perm, tree: ffc.DeviceTree, kernel: ffc.Kernel, precision=ffc.MIXED, s_probe: int = 512,
                   min_level: int = 2, stream=None, reps: int = 1, cache_path: str | None = None) -> dict:
    """One evaluation path for a tree call, timed where it runs: for every candidate, a compression call of a
    single sample-size round (s0 = s_max = s_probe, uniform rows) on the caller's tree with the tree profile
    on, after one untimed call; the candidate with the least evaluation-phase time (its prep and block
    kernels, CUDA events) wins. Single-block timings (``tune_eval``) carry a per-call overhead of the order
    of the small blocks' kernel time and cannot rank the paths at d = 128; the round holds the tree's real
    mix of block sizes. Keyed by (d, precision, kernel, N, depth, s_probe, point dtype) and cached."""
    if precision != ffc.MIXED or kernel.kind == ffc.LAPLACE:
        return {"eval_path": ffc.EVAL_DEFAULT, "source": "no choice"}
    N, d = points_perm.shape
    key = (f"tree:d={d},precision={precision},kernel={kernel.kind},N={N},depth={tree.depth},s={s_probe},"
           f"dtype={str(points_perm.dtype).split('.')[-1]}")
    if key not in _EVAL_CACHE and cache_path and os.path.exists(cache_path):
        with open(cache_path) as f:
            _EVAL_CACHE.update(json.load(f))
    if key in _EVAL_CACHE:
        return dict(_EVAL_CACHE[key], source="cache")
    kw = dict(tol=1e-6, precision=precision, s0=s_probe, s_max=s_probe, min_level=min_level, stream=stream)
    table = {}
    for path in EVAL_CANDIDATES:
        res = ffc.ffc_compress_tree(points_perm, tree, kernel, eval_path=path, **kw)   # untimed
        res.profile_enable(True)
        res.profile_reset()
        for _ in range(reps):
            res = ffc.ffc_compress_tree(points_perm, tree, kernel, eval_path=path, result=res, **kw)
        table[path] = res.profile()["ms"]["eval"] / reps
        res.close()
    best = min(table, key=table.get)
    out = {"eval_path": best, "eval_ms": round(table[best], 3), "s_probe": s_probe,
           "table": {str(k): round(v, 3) for k, v in table.items()}}
    _EVAL_CACHE[key] = out
    if cache_path:
        with open(cache_path, "w") as f:
            json.dump(_EVAL_CACHE, f, indent=1, sort_keys=True)
    return dict(out, source="measured")
