#!/usr/bin/env python
"""Benchmark: tree nodes compressed per second by sampled-row ID on one GB300.

Default configuration (the mixed-precision one): N = 262,144 points in d = 128
from a 16-component Gaussian mixture whose coordinate k has variance 1/k,
PCA median-split tree with leaf size 256 (levels 2..10, 2,044 nodes, n =
65,536 .. 256); one "step" compresses every node twice, once per kernel of
the configuration: Laplace |x - y|^-126 and the cubic polynomial
(x.y / 128 + 1)^3 (4,088 node compressions). Tolerance 1e-6 on
||R22||_F / ||K'||_F, s = 128 doubling to at most 2,048. Synthetic data; the
tree is built once on the GPU before timing (support).

Timing: W warm-up steps, then K timed steps, each bracketed by CUDA events
on the launching stream; a 512 MB buffer is written between steps to flush
the 129 MB L2 (outside the events). Clocks are sampled with nvidia-smi
during the timed steps. `value` is nodes / second over the timed steps;
`e2e` repeats the measurement through host buffers (pinned H2D of the
points and tree, compression, D2H of every node's rank, status, residual,
skeleton and interpolation matrix). `cpu_baseline` and `--impl reference`
time the FP64 oracle over a pool of single-threaded processes on the host
cores, each step one complete pass over a fixed seeded sample of nodes from
the tree's two deepest levels (the oracle's time for the largest nodes is
minutes each).

The timed form (`value`) is mixed precision with the learned row proposal,
whose network is first trained on the GPU (untimed) with the standard recipe
(leaves of the d = 128 and d = 1000 generators). Beside it: plain FP64 with
uniform sampling (`fp64_plain`, the reference point of the speedup), and the
other configurations (d = 16 and d = 1,000 trees) with their own plain FP64
arms (`extra_configs`). The oracle compresses with the uniform sampler (the
network's weights come from the GPU path and are never fed to the oracle).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

# One tree and kernel each ("parts"); a configuration compresses one or more parts per step.
WORKLOADS = {
    # N = 65,536 in d = 16, 8-component mixture, leaf 256 (levels 2..8, 508 nodes), Gaussian h = 2
    "c2": {"workload": "tree_compress_gaussian_mixture_N65536_d16", "gen": "gaussian_mixture", "N": 65536, "d": 16,
           "components": 8, "data_seed": 0, "leaf_size": 256, "kernel": "gaussian", "h": 2.0, "points": "f64"},
    # N = 262,144 in d = 128 with per-coordinate variance 1/k, leaf 256 (levels 2..10, 2,044 nodes)
    "c3-laplace": {"workload": "tree_compress_decaying_mixture_N262144_d128_laplace", "gen": "decaying_mixture",
                   "N": 262144, "d": 128, "components": 16, "data_seed": 1000, "leaf_size": 256, "kernel": "laplace",
                   "points": "f64"},
    "c3-poly": {"workload": "tree_compress_decaying_mixture_N262144_d128_poly3", "gen": "decaying_mixture",
                "N": 262144, "d": 128, "components": 16, "data_seed": 1000, "leaf_size": 256, "kernel": "polynomial",
                "h": 128.0, "c": 1.0, "p": 3, "points": "f64"},
    # N = 100,000 of intrinsic dimension 10 in d = 1,000 (FP32), leaf 512 (levels 2..8, 508 nodes),
    # Gaussian with h = the median pairwise distance
    "c4": {"workload": "tree_compress_low_intrinsic_N100000_d1000_gaussian", "gen": "low_intrinsic", "N": 100000,
           "d": 1000, "d_i": 10, "data_seed": 1000, "leaf_size": 512, "kernel": "gaussian", "h": "median",
           "points": "f32"},
}
CONFIGS = {
    "c3": {"workload": "tree_compress_decaying_mixture_N262144_d128_laplace_and_poly3",
           "parts": ["c3-laplace", "c3-poly"]},
    "c2": {"workload": WORKLOADS["c2"]["workload"], "parts": ["c2"]},
    "c4": {"workload": WORKLOADS["c4"]["workload"], "parts": ["c4"]},
    "c3-laplace": {"workload": WORKLOADS["c3-laplace"]["workload"], "parts": ["c3-laplace"]},
    "c3-poly": {"workload": WORKLOADS["c3-poly"]["workload"], "parts": ["c3-poly"]},
}
DEFAULT_CONFIG = "c3"
COMMON = {"tol": 1e-6, "s0": 128, "s_max": 2048, "min_level": 2, "xi": 1.0, "sample_seed": 0}
WORKLOAD = dict(WORKLOADS["c2"], **COMMON)


def select_workload(name: str):
    """Make part `name` the one the per-part helpers below describe."""
    global WORKLOAD
    WORKLOAD = dict(WORKLOADS[name], **COMMON)
    WORKLOAD["name"] = name


def workload_points(seed_offset: int = 0):
    """The workload's synthetic points (numpy, float64 or float32 as the workload stores them)."""
    import workloads
    W = WORKLOAD
    seed = W["data_seed"] + seed_offset
    if W["gen"] == "gaussian_mixture":
        return workloads.gaussian_mixture(N=W["N"], d=W["d"], k=W["components"], seed=seed)
    if W["gen"] == "decaying_mixture":
        return workloads.decaying_mixture(N=W["N"], d=W["d"], k=W["components"], seed=seed)
    return workloads.low_intrinsic(N=W["N"], d_i=W["d_i"], d_e=W["d"], seed=seed)


def workload_kernel(kernels_mod, P):
    """Kernel description for ``kernels_mod`` (the binding or the oracle) on the points P."""
    import workloads
    W = WORKLOAD
    kind = {"gaussian": "GAUSSIAN", "laplace": "LAPLACE", "polynomial": "POLYNOMIAL"}[W["kernel"]]
    code = getattr(kernels_mod, kind)
    h = W.get("h", 1.0)
    if h == "median":
        h = workloads.median_pairwise_distance(P)
    return kernels_mod.Kernel(code, h=float(h), c=float(W.get("c", 1.0)), p=int(W.get("p", 3)))


def kernel_label(h_value=None):
    W = WORKLOAD
    if W["kernel"] == "gaussian":
        return f"gaussian h={W['h'] if h_value is None else round(h_value, 6)}"
    if W["kernel"] == "laplace":
        return f"laplace |x-y|^-{W['d'] - 2}"
    return f"polynomial (x.y/{W['h']:g} + {W['c']:g})^{W['p']}"


def part_label(p):
    """Kernel label of a part's inputs."""
    select_workload(p.name)
    return kernel_label(p.kern.h)


def points_key(name):
    """Parts with the same points and leaf size share one tree."""
    W = WORKLOADS[name]
    return (W["gen"], W["N"], W["d"], W["data_seed"], W["leaf_size"])


METRIC = "nodes compressed/sec at ID rel. error <=1e-6; chosen form vs plain FP64 GPU"
UNIT = "nodes/s"


def _env_rank():
    return int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("LOCAL_RANK", "0"))


def load_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            return json.load(f), "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


# FP64 FMA rate of a GB300 (nominal 1.25 TFLOP/s dense FP64); the QR of the
# plain path is bound by it.
FP64_PEAK_TFLOPS = 1.25


class ClockSampler:
    """nvidia-smi clocks/throttle reasons every 200 ms while the timed region runs."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines: list[str] = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, FileNotFoundError):
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[3:7]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


class PartInputs:
    """One part's device inputs: points in tree order, the tree and the kernel (the points and tree are
    shared by parts with the same generator)."""

    def __init__(self, name, P, tree, Pp, kern):
        self.name, self.P, self.tree, self.Pp, self.kern = name, P, tree, Pp, kern


def build_config_inputs(torch, dev, cfg_name):
    from paper_1409_2802_gb300 import ffc
    rank, _, _ = _env_rank()
    shared = {}
    out = []
    for part in CONFIGS[cfg_name]["parts"]:
        select_workload(part)
        key = points_key(part)
        if key not in shared:
            P = workload_points(rank)
            Pd = torch.tensor(P, device=dev)
            tree = ffc.ffc_build_tree(Pd, WORKLOAD["leaf_size"])
            shared[key] = (P, tree, Pd[tree.perm].contiguous())
            del Pd
        P, tree, Pp = shared[key]
        out.append(PartInputs(part, P, tree, Pp, workload_kernel(ffc, P)))
    return out


def max_over_ranks(value: float, world: int, device="cpu") -> float:
    """The largest of the ranks' values (a job's time is its slowest rank's); all ranks get it."""
    if world <= 1:
        return float(value)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(nodes_per_rank: int, steps: int, world: int, max_ms: float) -> float:
    """Whole-job nodes/s: every rank compresses its own replica of the workload (weak scaling)."""
    return nodes_per_rank * steps * world / (max_ms / 1e3)


def precision_code(ffc, name):
    return ffc.FP64 if name == "fp64" else ffc.MIXED


def compress_kwargs():
    W = WORKLOAD
    return dict(tol=W["tol"], min_level=W["min_level"], s0=W["s0"], s_max=W["s_max"], xi=W["xi"],
                seed=W["sample_seed"])


def run_gpu_steps(torch, ffc, parts, precision, steps, warmup, flush_buf, stream, proposal=None, qr_kw=None,
                  sampler=None):
    """W warm-up and K timed steps; a step compresses every part's tree. Returns (results, per-step ms,
    profiles per part)."""
    qr_kw = qr_kw or {}
    results = {p.name: None for p in parts}

    def step():
        for p in parts:
            select_workload(p.name)
            prop = proposal[p.name] if isinstance(proposal, dict) else proposal
            results[p.name] = ffc.ffc_compress_tree(p.Pp, p.tree, p.kern, precision=precision, result=results[p.name],
                                                    stream=stream, proposal=prop, sampler=sampler,
                                                    **compress_kwargs(), **qr_kw.get(p.name, {}))

    for w in range(warmup):
        step()
        if w == 0:   # profile from the second warm-up step on, so its rounds' graphs are captured untimed
            for r in results.values():
                r.profile_enable(True)
    for r in results.values():
        r.profile_enable(True)
        r.profile_reset()
    times = []
    for _ in range(steps):
        flush_buf.fill_(1.0)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        step()
        e1.record(stream)
        e1.synchronize()
        times.append(e0.elapsed_time(e1))
    profs = {}
    for name, r in results.items():
        profs[name] = r.profile()
        r.profile_enable(False)
    return results, times, profs


def run_e2e(torch, ffc, parts, precision, steps, warmup, stream, proposal=None, qr_kw=None):
    """Same metric through host buffers: pinned H2D of the points and tree (once per step, shared by the
    parts), every part compressed, D2H of every node's outputs, every step."""
    dev = parts[0].Pp.device
    trees = {}
    for p in parts:
        if id(p.tree) not in trees:
            hP = p.Pp.cpu().pin_memory()
            th = {n: getattr(p.tree, n).cpu().pin_memory() for n in ("begin", "count", "centroid", "radius")}
            dP = torch.empty_like(hP, device=dev)
            dT = {n: torch.empty_like(v, device=dev) for n, v in th.items()}
            trees[id(p.tree)] = (hP, th, dP, dT, ffc.DeviceTree(p.tree.depth, p.tree.perm, dT["begin"], dT["count"],
                                                                dT["centroid"], dT["radius"]))
    h2d = sum(v[0].numel() * v[0].element_size() + sum(t.numel() * t.element_size() for t in v[1].values())
              for v in trees.values())
    results = {p.name: None for p in parts}
    d2h_bytes = []
    qr_kw = qr_kw or {}

    def step():
        with torch.cuda.stream(stream):
            for hP, th, dP, dT, _ in trees.values():
                dP.copy_(hP, non_blocking=True)
                for n in dT:
                    dT[n].copy_(th[n], non_blocking=True)
        nb = 0
        for p in parts:
            select_workload(p.name)
            _, _, dP, _, dtree = trees[id(p.tree)]
            prop = proposal[p.name] if isinstance(proposal, dict) else proposal
            results[p.name] = ffc.ffc_compress_tree(dP, dtree, p.kern, precision=precision, result=results[p.name],
                                                    stream=stream, proposal=prop, **compress_kwargs(),
                                                    **qr_kw.get(p.name, {}))
            with torch.cuda.stream(stream):
                v = ffc.tree_result_views(results[p.name])
                out = {kk: v[kk].to("cpu", non_blocking=False)
                       for kk in ("rank", "s", "status", "r22_rel", "skel", "T_off", "T")}
            nb += sum(t.numel() * t.element_size() for t in out.values())
        d2h_bytes.append(nb)

    for _ in range(warmup):
        step()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        step()
    e1.record(stream)
    e1.synchronize()
    wall = time.perf_counter() - t0
    ms = e0.elapsed_time(e1)
    n_nodes = sum(ffc.tree_result_views(r)["n_out"] for r in results.values())
    for r in results.values():
        r.close()
    return {"value": n_nodes * steps / (ms / 1e3), "unit": UNIT, "h2d_bytes_per_step": int(h2d),
            "d2h_bytes_per_step": int(statistics.mean(d2h_bytes[-steps:])), "wall_s": wall, "steps": steps}


# --------------------------------------------------------------------------- oracle legs

def oracle_sample(cfg_name, per_part=16, seed=12345):
    """The fixed node sample of the oracle legs: per part, `per_part` seeded nodes of the tree's two deepest
    levels (node ids depend only on N and the leaf size), largest first."""
    import numpy as np
    from oracle import tree as o_tree
    out = []
    for part in CONFIGS[cfg_name]["parts"]:
        W = WORKLOADS[part]
        D = o_tree.tree_depth(W["N"], W["leaf_size"])
        cand = np.arange((1 << (D - 1)) - 1, (1 << (D + 1)) - 1)
        pick = np.random.default_rng(seed).choice(cand, min(per_part, cand.size), replace=False)
        out += [(part, int(nd)) for nd in sorted(pick.tolist())]
    return out


def oracle_compress(state, part, node):
    from oracle import compress as o_compress
    Pp, t, kernel = state[part]
    W = dict(WORKLOADS[part], **COMMON)
    return o_compress.compress_node(Pp, t, int(node), kernel, W["tol"], W["sample_seed"], W["s0"], W["s_max"],
                                    W["xi"])


_WORKER = {}


def _worker_init(cfg_name):
    """Pool worker: the oracle's inputs of every part (parts with the same points share the tree)."""
    from oracle import kernels as o_kernels
    from oracle import tree as o_tree
    state, trees = {}, {}
    for part in CONFIGS[cfg_name]["parts"]:
        select_workload(part)
        key = points_key(part)
        if key not in trees:
            P = workload_points()
            t = o_tree.build_tree(P, WORKLOAD["leaf_size"])
            trees[key] = (P, P[t.perm].astype("float64"), t)
        P, Pp, t = trees[key]
        state[part] = (Pp, t, workload_kernel(o_kernels, P))
    _WORKER["state"] = state


def _worker_compress(item):
    part, node = item
    oracle_compress(_WORKER["state"], part, node)
    return item


class OraclePool:
    """The FP64 oracle over a pool of single-threaded processes (spawned, so that no GPU state is
    forked); each pass compresses a fixed list of (part, node) items completely."""

    def __init__(self, cfg_name: str, workers: int):
        import multiprocessing as mp
        self.workers = max(1, int(workers))
        self.cfg = cfg_name
        ctx = mp.get_context("spawn")
        for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
            os.environ[k] = "1"
        self.pool = ctx.Pool(self.workers, initializer=_worker_init, initargs=(cfg_name,))
        # every worker holds its inputs before the first timed pass
        self.pool.map(_noop, range(self.workers), chunksize=1)

    def run_pass(self, items) -> float:
        t0 = time.perf_counter()
        for _ in self.pool.imap_unordered(_worker_compress, items, chunksize=1):
            pass
        return time.perf_counter() - t0

    def close(self):
        self.pool.terminate()
        self.pool.join()


def _noop(i):
    return i


def host_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def sample_label(items, workers):
    parts = sorted({p for p, _ in items})
    return (f"{len(items)} nodes ({', '.join(f'{sum(1 for q, _ in items if q == p)} of {p}' for p in parts)}), "
            f"a seeded sample of the two deepest tree levels, each pass compressing all of them; "
            f"{workers} single-threaded processes (OMP/OpenBLAS = 1), uniform sampler")


def cpu_baseline_leg(cfg_name, workers, min_seconds=10.0) -> dict:
    """The oracle on the host cores after the GPU work: complete passes over the fixed sample until at
    least `min_seconds` have gone by; nodes / second."""
    items = oracle_sample(cfg_name)
    pool = OraclePool(cfg_name, workers)
    try:
        el, done, passes = 0.0, 0, 0
        while el < min_seconds or passes == 0:
            el += pool.run_pass(items)
            done += len(items)
            passes += 1
    finally:
        pool.close()
    return {"value": done / el, "unit": UNIT, "cores": pool.workers, "kind": "oracle",
            "sample": sample_label(items, pool.workers) + f"; {passes} passes in {el:.1f} s"}


def reference_arm(args, rank, world):
    """--impl reference: the FP64 CPU oracle; each step is one complete pass over the fixed sample."""
    if rank != 0:
        return 0
    items = oracle_sample(args.workload)
    try:
        pool = OraclePool(args.workload, args.cpu_workers or host_cores())
    except (OSError, RuntimeError) as e:
        print(json.dumps({"impl": "reference", "unavailable": f"oracle pool failed: {e}"}))
        return 0
    try:
        for _ in range(args.warmup):
            pool.run_pass(items)
        times = [pool.run_pass(items) for _ in range(args.steps)]
    finally:
        pool.close()
    el = sum(times)
    value = len(items) * args.steps / el
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 0, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": el * 1e3 / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": config_block(args.workload, "fp64", "uniform"),
        "cpu_baseline": {"value": value, "unit": UNIT, "kind": "oracle", "cores": pool.workers,
                         "sample": sample_label(items, pool.workers)},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


def config_block(cfg_name, precision, sampler, extra=None):
    parts = CONFIGS[cfg_name]["parts"]
    W0 = dict(WORKLOADS[parts[0]], **COMMON)
    cfg = {"workload": CONFIGS[cfg_name]["workload"], "precision": precision, "sampler": sampler,
           "parts": parts, "N": W0["N"], "d": W0["d"], "leaf_size": W0["leaf_size"], "points": W0["points"],
           "tol": W0["tol"], "s": "128 doubling to 2048", "l2": "flushed between steps (512 MB write)"}
    if extra:
        cfg.update(extra)
    return cfg


FP32_PEAK_TFLOPS = 80.5   # 152 SMs x 128 FP32 lanes x 2 flops x 2.07 GHz (nominal)



def qr_traffic(precision_name, sampler, shape=None, workload_name=None):
    """DRAM bytes per step of the QR launches from the committed ncu record, while the kernel source
    and the QR launch shape (``shape``: qr_big_min_s / qr_l2_budget_mb, None = the library defaults)
    still match the ones the counters were taken on; else None."""
    import glob
    import hashlib
    src = os.path.join(ROOT, "paper_1409_2802_gb300", "csrc", "cpqr.cu")
    with open(src, "rb") as f:
        h = hashlib.sha256(f.read()).hexdigest()
    for path in glob.glob(os.path.join(ROOT, "profiles", "cpqr_traffic_*.md")):
        rec = {}
        with open(path) as f:
            for line in f:
                if ":" in line and not line.startswith(("#", "|", "*", " ")):
                    k, v = line.split(":", 1)
                    rec[k.strip()] = v.strip()
        want = dict(shape or {"qr_big_min_s": 1024, "qr_l2_budget_mb": 96})
        same_shape = all(str(want.get(k_)) == rec.get(k_) for k_ in ("qr_big_min_s", "qr_l2_budget_mb"))
        if (rec.get("cpqr_sha256") == h and rec.get("workload") == (workload_name or WORKLOAD["workload"])
                and rec.get("precision") == precision_name and rec.get("sampler") == sampler and same_shape):
            return float(rec["traffic_bytes_per_step"]), os.path.relpath(path, ROOT)
    return None, None


def eval_roofline(prof, steps, precision_name, peaks, peak_src):
    """The block evaluation as a GEMM: 2 s n d flops per block (the library counts the direct form's
    3 s n d, or 2 s n d for the polynomial). Mixed precision at d >= 64 (Gaussian, polynomial) runs on
    the tensor cores with six BF16 partial products per multiply-add; the rest is SIMT."""
    W = WORKLOAD
    ms = prof["ms"]["eval"] / max(steps, 1)
    per_coord = 2.0 if W["kernel"] == "polynomial" else 3.0
    gemm = prof["eval_flops"] / per_coord * 2.0 / max(steps, 1)
    tflops = gemm / (ms / 1e3) / 1e12 if ms > 0 else 0.0
    tensor = precision_name == "mixed" and W["kernel"] != "laplace" and W["d"] >= 64
    if tensor:
        # timed inside a long step: the sustained figure
        peak = peaks.get("bf16_tflops_sustained", peaks.get("bf16_tflops", 1710.8))
        return {"kernel": "tc5_kernel (tcgen05.mma, TMEM accumulators, TMA-staged split-BF16 planes, FP32 "
                          "accumulate; with its plane-prep kernel)", "bound": "tensor",
                "achieved": tflops, "peak": peak, "unit": "TFLOP/s", "frac": tflops / peak,
                "tensor_work_tflops": 6.0 * tflops, "tensor_work_frac": 6.0 * tflops / peak,
                "peak_source": f"{peak_src} dense BF16, sustained (MEASURED_PEAKS.json bf16_tflops_sustained, "
                               "tcgen05 cuBLAS)",
                "gemm_flops_per_step": gemm, "ms_per_step": ms}
    peak, src = alu_peak(peaks, precision_name)
    return {"kernel": "eval_kernel (SIMT)", "bound": "alu", "achieved": tflops, "peak": peak, "unit": "TFLOP/s",
            "frac": tflops / peak, "gemm_flops_per_step": gemm, "ms_per_step": ms, "peak_source": src}


def alu_peak(peaks, precision_name):
    """FP32 (mixed) or FP64 ALU peak: the one measured in this run when present, else nominal."""
    key = "fp64_tflops" if precision_name == "fp64" else "fp32_tflops"
    if peaks.get(key):
        return peaks[key], f"measured in this run: {peaks.get(key + '_how', '')}"
    if precision_name == "fp64":
        return FP64_PEAK_TFLOPS, "nominal FP64 rate of GB300"
    return FP32_PEAK_TFLOPS, "nominal FP32 rate of GB300 (152 SMs x 128 lanes x 2 flops x 2.07 GHz)"


def measure_alu_peaks(torch, dev):
    """FP64 and FP32 (TF32 off) GEMM throughput of this GPU (cuBLAS through torch.matmul, best of 3 after a
    warm-up): the denominators of the ALU fractions of the FP64 and FP32 paths."""
    out = {}
    prev = torch.backends.cuda.matmul.allow_tf32
    torch.backends.cuda.matmul.allow_tf32 = False
    try:
        for key, dt, n in (("fp64_tflops", torch.float64, 8192), ("fp32_tflops", torch.float32, 8192)):
            a = torch.randn(n, n, dtype=dt, device=dev)
            b = torch.randn(n, n, dtype=dt, device=dev)
            torch.matmul(a, b)
            best = float("inf")
            for _ in range(3):
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record()
                torch.matmul(a, b)
                e1.record()
                e1.synchronize()
                best = min(best, e0.elapsed_time(e1))
            out[key] = 2.0 * n ** 3 / (best / 1e3) / 1e12
            out[key + "_how"] = f"torch.matmul {str(dt).replace('torch.', '')} {n}^3, best of 3 (TF32 off)"
            del a, b
    finally:
        torch.backends.cuda.matmul.allow_tf32 = prev
    torch.cuda.empty_cache()
    return out


def combine_profiles(profs):
    """Sum of the per-part profiles of one arm."""
    keys = ("sample", "eval", "qr", "trsm", "bookkeeping")
    out = {"ms": {k: sum(p["ms"][k] for p in profs) for k in keys},
           "launches": sum(p["launches"] for p in profs), "qr_launches": sum(p["qr_launches"] for p in profs)}
    for k in ("qr_flops", "eval_flops", "qr_bytes"):
        out[k] = sum(p[k] for p in profs)
    out["qr_ms_round"] = [sum(p["qr_ms_round"][i] for p in profs) for i in range(8)]
    out["items_round"] = [sum(p["items_round"][i] for p in profs) for i in range(8)]
    return out


def qr_roofline(prof, steps, precision_name, peaks, peak_src, sampler="learned", shape=None, workload_name=None):
    """Roofline of the pivoted QR from the library's live per-phase CUDA-event timing (all parts of a step).

    Algorithmic bytes: one read and one write of every sampled block K' (s x n)
    per QR launch. The Householder QR streams the trailing matrix once per step,
    (s - k)(n - k) elements at step k; that volume is reported as `streamed_gbs`,
    and the FP32/FP64 ALU rate beside it.
    """
    phase_ms = prof["ms"]
    qr_ms = phase_ms["qr"] / max(steps, 1)
    esz = 8.0 if precision_name == "fp64" else 4.0
    tflops = prof["qr_flops"] / steps / (qr_ms / 1e3) / 1e12 if qr_ms > 0 else 0.0
    gbs = prof["qr_bytes"] / steps / (qr_ms / 1e3) / 1e9 if qr_ms > 0 else 0.0
    streamed = prof["qr_flops"] / 2.0 * esz / steps / (qr_ms / 1e3) / 1e9 if qr_ms > 0 else 0.0
    hbm = peaks.get("hbm_gbs", 6775.3)
    apk, src = alu_peak(peaks, precision_name)
    kern = ("cpqr_kernel<double> (pivoted QR, FP64)" if precision_name == "fp64"
            else "cpqr_kernel<float> (pivoted QR, FP32 updates, FP64 norms)")
    traffic, traffic_src = qr_traffic(precision_name, sampler, shape, workload_name)
    return {
        "kernel": kern, "bound": "hbm", "achieved": gbs, "peak": hbm, "unit": "GB/s", "frac": gbs / hbm,
        "traffic": traffic, "traffic_unit": "bytes per step (all QR launches of one call)",
        "traffic_source": traffic_src,
        "peak_source": f"{peak_src} HBM copy bandwidth (MEASURED_PEAKS.json hbm_gbs)",
        "streamed_gbs": streamed, "streamed_frac": streamed / hbm,
        "alu": {"achieved": tflops, "peak": apk, "unit": "TFLOP/s", "frac": tflops / apk, "source": src},
        "dominant_phase": max(phase_ms, key=phase_ms.get),
        "phase_ms_per_step": {k: v / steps for k, v in phase_ms.items()},
        "qr_ms_per_step_by_round": [round(v / steps, 3) for v in prof.get("qr_ms_round", [])],
        "nodes_per_step_by_round": [int(v // steps) for v in prof.get("items_round", [])],
        "qr_flops_per_step": prof["qr_flops"] / steps, "qr_bytes_per_step": prof["qr_bytes"] / steps,
    }


def trsm_roofline(ffc, results, trsm_ms_per_step, peaks, precision_name="fp64"):
    """The triangular solve T = R11^-1 R12: r^2 (n - r) algorithmic flops per node (one multiply-add per
    entry of R11 above the diagonal and column of R12, counted as 2 flops over half the triangle), from the
    final ranks of every node of every part.
    * FP64 path: the blocked FP64 back-substitution, against the measured FP64 peak.
    * Mixed path: two FP32 solves and a double-float residual (9 FP32 operations per term), about 11 FP32
      operations per algorithmic multiply-add; against the measured FP32 peak, counting those operations
      (`executed_tflops`), and beside the FP64 peak the plain solve is bound by (`vs_fp64_peak`)."""
    flops = 0.0
    for res in results:
        h = ffc.tree_result_to_host(res)
        r = h["rank"].astype("float64")
        n = (h["skel_off"][1:] - h["skel_off"][:-1]).astype("float64")
        flops += float((r * r * (n - r)).sum())
    tf = flops / (trsm_ms_per_step / 1e3) / 1e12 if trsm_ms_per_step > 0 else 0.0
    p64, src64 = alu_peak(peaks, "fp64")
    if precision_name != "mixed":
        return {"kernel": "trsm_kernel (blocked back-substitution, FP64)", "bound": "alu", "achieved": tf,
                "peak": p64, "unit": "TFLOP/s", "frac": tf / p64, "flops_per_step": flops,
                "ms_per_step": trsm_ms_per_step, "peak_source": src64}
    p32, src32 = alu_peak(peaks, "mixed")
    executed = tf * 11.0 / 2.0   # FP32 operations per algorithmic flop (2 flops per multiply-add)
    return {"kernel": "trsm_refine_kernel (FP32 solves refined once, double-float residual)", "bound": "alu",
            "achieved": executed, "peak": p32, "unit": "TFLOP/s", "frac": executed / p32,
            "algorithmic_tflops": tf, "vs_fp64_peak": tf / p64, "flops_per_step": flops,
            "ms_per_step": trsm_ms_per_step, "peak_source": src32, "fp64_peak_source": src64}


def timed_call(torch, stream, fn, reps=2):
    """Milliseconds of the last of `reps` calls of fn() on `stream` (CUDA events), and its result."""
    out = None
    ms = 0.0
    for _ in range(reps):
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        out = fn()
        e1.record(stream)
        e1.synchronize()
        ms = e0.elapsed_time(e1)
    return ms, out


def d16_studies(torch, ffc, part, prop, stream, prec):
    """On the d = 16 tree (untimed in the headline): the paper's samplers beside the learned one at equal s,
    nested skeletonization, and the evaluation of the potential from the representations."""
    import numpy as np
    out = {}
    W = dict(WORKLOADS[part.name], **COMMON)
    select_workload(part.name)
    # (1) samplers at equal s: every node sampled with s = 256 rows (rank cap 128), mixed precision
    s_eq = 256
    samplers = {"uniform": (ffc.SAMPLE_UNIFORM, None), "learned": (None, prop),
                "distance": (ffc.SAMPLE_DISTANCE, None), "inverse_distance": (ffc.SAMPLE_INV_DISTANCE, None),
                "nearest_neighbours": (ffc.SAMPLE_NEAREST, None)}
    sam = {}
    for name, (code, pr) in samplers.items():
        kw = dict(tol=W["tol"], min_level=W["min_level"], s0=s_eq, s_max=s_eq, xi=W["xi"], seed=W["sample_seed"])
        ms, res = timed_call(torch, stream, lambda: ffc.ffc_compress_tree(part.Pp, part.tree, part.kern,
                                                                          precision=prec, stream=stream, proposal=pr,
                                                                          sampler=code, **kw))
        n = int(ffc.tree_result_views(res)["n_out"])
        e = arm_errors(torch, ffc, part.Pp, part.tree, part.kern, res)
        ee = np.asarray(e["errors"])
        sam[name] = {"nodes_per_s": n / (ms / 1e3), "ms_per_call": ms, "median_full_block_error": float(np.median(ee)),
                     "max_full_block_error": float(ee.max()), "fraction_at_or_below_1e-6": float(np.mean(ee <= 1e-6)),
                     "mean_rank": e["mean_rank"]}
        res.close()
    out["samplers_at_equal_s"] = {"s": s_eq, "precision": "mixed" if prec == ffc.MIXED else "fp64",
                                  "nodes_checked": 12, "note": "leverage sampling needs the full block's SVD "
                                  "(n <= 1024) and is compared single-node in the tests", "by_sampler": sam}
    # (2) nested skeletonization against the plain form, same sampler (learned) and tolerance
    kw = compress_kwargs()
    nest = {}
    for label, nested in (("plain", False), ("nested", True)):
        ms, res = timed_call(torch, stream, lambda: ffc.ffc_compress_tree(part.Pp, part.tree, part.kern,
                                                                          precision=prec, stream=stream,
                                                                          proposal=prop, nested=nested, **kw))
        h = ffc.tree_result_to_host(res)
        nest[label] = {"nodes_per_s": len(h["node"]) / (ms / 1e3), "ms_per_call": ms,
                       "mean_columns": float(h["ncols"].mean()), "mean_rank": float(h["rank"].mean())}
        if label == "nested":
            # (3) the potential at every point from the nested representations, against the direct sum
            q = torch.as_tensor(np.random.default_rng(11).standard_normal(part.Pp.shape[0])).to(part.Pp.device)
            ms_s, (u_s, _) = timed_call(torch, stream, lambda: ffc.ffc_tree_apply(part.Pp, part.tree, res, q,
                                                                                  mode=ffc.APPLY_SKELETON,
                                                                                  stream=stream))
            ms_d, (u_d, _) = timed_call(torch, stream, lambda: ffc.ffc_tree_apply(part.Pp, part.tree, res, q,
                                                                                  mode=ffc.APPLY_DIRECT,
                                                                                  stream=stream))
            err = float(torch.linalg.vector_norm(u_s - u_d) / torch.linalg.vector_norm(u_d))
            npts = int(part.Pp.shape[0])
            out["apply"] = {"targets": npts, "skeleton_ms": ms_s, "direct_ms": ms_d,
                            "targets_per_s_skeleton": npts / (ms_s / 1e3), "targets_per_s_direct": npts / (ms_d / 1e3),
                            "relative_error_vs_direct": err, "representation": "nested, learned rows, mixed",
                            "what": "potential at every point: far field from the outgoing representations, near "
                                    "leaves direct (ffc_tree_apply)"}
        res.close()
    out["nested_skeletonization"] = nest
    return out


def arm_errors(torch, ffc, Pp, tree, k, res, n_sample=12, seed=7, max_n=4096):
    """Full-block ID error of a seeded sample of nodes of one arm's result (outside the timed region): nodes
    of at most max_n sources (the FP64 error of a 65,536-source node against its whole far field takes
    seconds)."""
    import numpy as np
    W = WORKLOAD
    h = ffc.tree_result_to_host(res)
    v = ffc.tree_result_views(res)
    nodes = h["node"]
    begin, count = tree.begin.cpu().numpy(), tree.count.cpu().numpy()
    cand = np.flatnonzero(count[nodes] <= max_n)
    pick = sorted(np.random.default_rng(seed).choice(cand, min(n_sample, cand.size), replace=False).tolist())
    errs = []
    for i in pick:
        node = int(nodes[i])
        b, n = int(begin[node]), int(count[node])
        far = ffc.ffc_far_field(Pp, x_c=tree.centroid[node].contiguous(), radius=float(tree.radius[node]), xi=W["xi"],
                                ex_begin=b, ex_end=b + n)
        r = int(h["rank"][i])
        skel = v["skel"][int(h["skel_off"][i]): int(h["skel_off"][i]) + n]
        off = int(h["T_off"][i])
        T = v["T"][off: off + r * (n - r)].view(n - r, r).t() if r else torch.zeros((0, n), device=Pp.device,
                                                                                      dtype=torch.float64)
        errs.append(ffc.ffc_id_error(k, Pp, Pp[b:b + n], skel, T, r, rows=far))
    return {"nodes": [int(nodes[i]) for i in pick], "errors": errs, "mean_rank": float(h["rank"].mean()),
            "mean_s": float(h["s"].mean()), "max_sources": int(max_n)}


def accuracy_summary(per_arm):
    """Per-arm error statistics; for each pair of arms that differ only in precision (same sampler, hence
    the same rows), the largest |e_mixed - e_fp64| is the reading of the accuracy gate
    |e_mixed - e_oracle| <= 1e-6: the FP64 GPU path equals the oracle's ID on the same rows (tests), so it
    stands in for the oracle here."""
    import numpy as np
    out = {"nodes_checked": next(iter(per_arm.values()))["nodes"]}
    for p, a in per_arm.items():
        e = np.asarray(a["errors"])
        out[p] = {"median_full_block_error": float(np.median(e)), "max_full_block_error": float(e.max()),
                  "nodes_checked": int(e.size), "nodes_at_or_below_1e-6": int(np.sum(e <= 1e-6)),
                  "fraction_at_or_below_1e-6": float(np.mean(e <= 1e-6)),
                  "nodes_at_or_below_1e-5": int(np.sum(e <= 1e-5)), "mean_rank": a["mean_rank"],
                  "mean_s": a["mean_s"]}
    for samp in ("learned", "uniform"):
        a, b = f"mixed_{samp}", f"fp64_{samp}"
        if a in per_arm and b in per_arm:
            dmax = float(max(abs(x - y) for x, y in zip(per_arm[a]["errors"], per_arm[b]["errors"])))
            out[f"max_abs_diff_mixed_vs_fp64_{samp}"] = dmax
            out[f"within_1e-6_{samp}"] = dmax <= 1e-6
    return out


def tune_parts(ffc, parts, prec, stream, proposal, max_step_s=1.5):
    """The launch shapes per part from the project's autotuner (untimed): the evaluation path (timed on single
    blocks of the tree's node sizes, cheap) always; the QR launch shape unless a part's single call takes
    longer than max_step_s (that part keeps the library's QR defaults: tuning would cost minutes)."""
    from paper_1409_2802_gb300 import autotune
    import torch
    kw, info = {}, {}
    for p in parts:
        select_workload(p.name)
        W = dict(WORKLOADS[p.name], **COMMON)
        te = autotune.tune_tree_eval(p.Pp, p.tree, p.kern, prec, min_level=W["min_level"], stream=stream)
        kw[p.name] = {"eval_path": te["eval_path"]}
        prop = proposal[p.name] if isinstance(proposal, dict) else proposal
        t0 = time.perf_counter()
        r = ffc.ffc_compress_tree(p.Pp, p.tree, p.kern, precision=prec, stream=stream, proposal=prop,
                                  **compress_kwargs())
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        r.close()
        if dt > max_step_s:
            info[p.name] = {"source": f"library defaults (one call takes {dt:.1f} s, too long to tune here)",
                            "eval": te}
            continue
        try:
            t = autotune.tune_tree(p.Pp, p.tree, p.kern, precision=prec, stream=stream, proposal=prop,
                                   eval_path=te["eval_path"], **compress_kwargs())
            kw[p.name].update({k_: t[k_] for k_ in ("qr_big_min_s", "qr_l2_budget_mb")})
            info[p.name] = dict(t, source="autotune", eval=te)
        except ffc.FFCError as e:
            info[p.name] = {"source": f"library defaults (autotune failed: {e})", "eval": te}
    return kw, info


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default=DEFAULT_CONFIG, choices=sorted(CONFIGS),
                    help="c3 (default): d = 128, Laplace and polynomial; c2: d = 16; c4: d = 1000 FP32; "
                         "c3-laplace / c3-poly: one kernel of c3")
    ap.add_argument("--precision", default="mixed", choices=["fp64", "mixed"],
                    help="precision of the timed form (value)")
    ap.add_argument("--sampler", default="learned", choices=["learned", "uniform"],
                    help="row sampler of the timed form; learned trains the proposal first (untimed)")
    ap.add_argument("--train-epochs", type=int, default=30)
    ap.add_argument("--train-nodes", type=int, default=100, help="training leaves per generator (d=128, d=1000)")
    ap.add_argument("--arm-steps", type=int, default=2, help="timed steps of the plain FP64 arm and other arms")
    ap.add_argument("--no-fp64-compare", action="store_true", help="skip the plain FP64 uniform arm")
    ap.add_argument("--all-arms", action="store_true", help="also time mixed + uniform and FP64 + learned")
    ap.add_argument("--no-extra-configs", action="store_true", help="skip the other configurations")
    ap.add_argument("--no-accuracy", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=10.0)
    ap.add_argument("--cpu-workers", type=int, default=0,
                    help="oracle processes of the CPU baseline and the reference arm (0 = every host core)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-autotune", action="store_true",
                    help="skip the QR launch-shape autotuner (untimed, before the timed form's steps)")
    args = ap.parse_args()

    rank, world, local = _env_rank()
    if args.impl == "reference":
        return reference_arm(args, rank, world)

    import torch
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    import workloads
    from paper_1409_2802_gb300 import ffc, learned
    ffc.lib()
    peaks, peak_src = load_peaks()
    peaks = dict(peaks, **measure_alu_peaks(torch, dev))
    params, train_info = None, None
    if args.sampler == "learned":
        params, train_info = learned.train_standard(seed=0, epochs=args.train_epochs,
                                                    nodes_per_generator=args.train_nodes, device=dev)
        torch.cuda.empty_cache()

    def proposal_for(parts):
        if params is None:
            return None
        return {p.name: (params, torch.as_tensor(workloads.projections(WORKLOADS[p.name]["d"], seed=7)).to(dev))
                for p in parts}

    stream = torch.cuda.Stream(device=dev)
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    prec = precision_code(ffc, args.precision)
    arm = f"{args.precision}_{args.sampler}"

    def timed(parts, prec_code, steps, warmup, prop, kw=None):
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()
        res, times, profs = run_gpu_steps(torch, ffc, parts, prec_code, steps, warmup, flush, stream, proposal=prop,
                                          qr_kw=kw)
        torch.cuda.synchronize()
        total = max_over_ranks(sum(times), world, dev)
        if world > 1:
            torch.distributed.barrier()
        return res, total, profs

    def n_nodes_of(res):
        return sum(int(ffc.tree_result_views(r)["n_out"]) for r in res.values())

    def close_all(res):
        for r in res.values():
            r.close()

    # ------------------------------------------------------------------ the headline configuration
    parts = build_config_inputs(torch, dev, args.workload)
    prop = proposal_for(parts)
    qr_kw, tune_info = ({}, {p.name: {"source": "library defaults"} for p in parts}) if args.no_autotune else \
        tune_parts(ffc, parts, prec, stream, prop)
    clocks = ClockSampler(local)
    clocks.start()
    res, total_ms, profs = timed(parts, prec, args.steps, args.warmup, prop, qr_kw)
    clk = clocks.stop()
    n_nodes = n_nodes_of(res)
    value = job_throughput(n_nodes, args.steps, world, total_ms)
    prof = combine_profiles(list(profs.values()))
    roof = qr_roofline(prof, args.steps, args.precision, peaks, peak_src, args.sampler, None,
                       CONFIGS[args.workload]["workload"])
    evals = {}
    for p in parts:
        select_workload(p.name)
        evals[p.name] = eval_roofline(profs[p.name], args.steps, args.precision, peaks, peak_src)
    roof["eval"] = evals
    roof["trsm"] = trsm_roofline(ffc, list(res.values()), prof["ms"]["trsm"] / args.steps, peaks, args.precision)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64" if prec == ffc.FP64 else "f32+f64", "data": "synthetic",
        "config": config_block(args.workload, args.precision, args.sampler,
                               {"nodes_per_step": n_nodes, "parallelism": f"replicas x{world}",
                                "kernels": {p.name: part_label(p) for p in parts}}),
        "clocks": clk, "gpu_launches": int(prof["launches"]), "roofline": roof,
    }
    if train_info is not None:
        line["config"]["proposal_training"] = train_info
    line["config"]["qr_launch_shape"] = tune_info
    errors = {p.name: {} for p in parts}
    if not args.no_accuracy and rank == 0:
        for p in parts:
            select_workload(p.name)
            errors[p.name][arm] = arm_errors(torch, ffc, p.Pp, p.tree, p.kern, res[p.name])
    close_all(res)
    del res
    # the plain FP64 GPU path on the same configuration (the speedup's reference point), and the other arms
    if not args.no_fp64_compare:
        arms = [("fp64", "uniform")]
        if args.all_arms and args.sampler == "learned":
            arms += [("mixed", "uniform"), ("fp64", "learned")]
        other = {}
        for pname, sname in arms:
            key = f"{pname}_{sname}"
            if key == arm:
                continue
            r_, ms_, pf_ = timed(parts, precision_code(ffc, pname), args.arm_steps, 1,
                                 prop if sname == "learned" else None)
            v_ = job_throughput(n_nodes, args.arm_steps, world, ms_)
            cp = combine_profiles(list(pf_.values()))
            other[key] = {"value": v_, "unit": UNIT, "ms_per_step": ms_ / args.arm_steps, "steps": args.arm_steps,
                          "warmup": 1, "phase_ms_per_step": {k: v / args.arm_steps for k, v in cp["ms"].items()},
                          "qr_roofline_frac": qr_roofline(cp, args.arm_steps, pname, peaks, peak_src, sname)["frac"]}
            if not args.no_accuracy and rank == 0:
                for p in parts:
                    select_workload(p.name)
                    errors[p.name][key] = arm_errors(torch, ffc, p.Pp, p.tree, p.kern, r_[p.name])
            close_all(r_)
            del r_
        if "fp64_uniform" in other:
            line["fp64_plain"] = other.pop("fp64_uniform")
            line["speedup_vs_fp64"] = value / line["fp64_plain"]["value"]
        if other:
            line["arms"] = other
    if not args.no_accuracy and rank == 0:
        line["accuracy"] = {name: accuracy_summary(e) for name, e in errors.items() if e}
    if not args.no_e2e:
        line["e2e"] = run_e2e(torch, ffc, parts, prec, max(2, min(3, args.steps)), 1, stream, proposal=prop,
                              qr_kw=qr_kw)
    del parts
    torch.cuda.empty_cache()
    # ------------------------------------------------------------------ the other configurations
    if not args.no_extra_configs and args.workload == DEFAULT_CONFIG:
        extra = {}
        for cname in ("c2", "c4"):
            cparts = build_config_inputs(torch, dev, cname)
            cprop = proposal_for(cparts)
            r1, ms1, pf1 = timed(cparts, prec, args.arm_steps, 1, cprop)
            nn = n_nodes_of(r1)
            close_all(r1)
            v1 = job_throughput(nn, args.arm_steps, world, ms1)
            ent = {"workload": CONFIGS[cname]["workload"], "value": v1, "unit": UNIT, "steps": args.arm_steps,
                   "warmup": 1, "ms_per_step": ms1 / args.arm_steps, "nodes_per_step": nn,
                   "phase_ms_per_step": {k: v / args.arm_steps for k, v in combine_profiles(list(pf1.values()))["ms"].items()}}
            if not args.no_fp64_compare:
                r2, ms2, _ = timed(cparts, ffc.FP64, args.arm_steps, 1, None)
                close_all(r2)
                v2 = job_throughput(nn, args.arm_steps, world, ms2)
                ent["fp64_plain"] = {"value": v2, "ms_per_step": ms2 / args.arm_steps, "steps": args.arm_steps}
                ent["speedup_vs_fp64"] = v1 / v2
            if cname == "c2" and rank == 0:
                try:   # auxiliary (untimed) studies: a failure there is recorded, not fatal to the line
                    ent["studies"] = d16_studies(torch, ffc, cparts[0], cprop[cparts[0].name] if cprop else None,
                                                 stream, prec)
                except Exception as e:   # noqa: BLE001
                    ent["studies"] = {"error": f"{type(e).__name__}: {str(e)[:200]}"}
            extra[cname] = ent
            del cparts
            torch.cuda.empty_cache()
        line["extra_configs"] = extra
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        try:
            line["cpu_baseline"] = cpu_baseline_leg(args.workload, args.cpu_workers or host_cores(), args.cpu_seconds)
        except (OSError, RuntimeError) as e:
            line["cpu_baseline"] = {"value": None, "unit": UNIT, "kind": "oracle", "cores": 0,
                                    "sample": f"oracle pool failed: {e}"}
    if rank == 0:
        print(json.dumps(line))
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
