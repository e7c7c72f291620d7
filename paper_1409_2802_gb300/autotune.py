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
"""
from __future__ import annotations

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
