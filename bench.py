#!/usr/bin/env python
"""Benchmark: tree nodes compressed per second by sampled-row ID on one GB300.

Workload (one "step" = one full ffc_compress_tree call over every node at
level >= 2): N = 65,536 points in d = 16 from an 8-component Gaussian mixture
(means uniform in [-5, 5]^16, sigma 1), PCA median-split tree with leaf size
256 (levels 2..8, 508 nodes, n = 16,384 .. 256), Gaussian kernel h = 2,
tolerance 1e-6 on ||R22||_F / ||K'||_F, s = 128 doubling to at most 2,048.
Synthetic data; the tree is built once on the GPU before timing (support).

Timing: W warm-up steps, then K timed steps, each bracketed by CUDA events
on the launching stream; a 512 MB buffer is written between steps to flush
the 129 MB L2 (outside the events). Clocks are sampled with nvidia-smi
during the timed steps. `value` is nodes / second over the timed steps;
`e2e` repeats the measurement through host buffers (pinned H2D of the
permuted points and tree, compression, D2H of every node's rank, status,
residual, skeleton and interpolation matrix). `cpu_baseline` times the FP64
oracle on a seeded, time-bounded sample of the same nodes in a
single-threaded subprocess; `--impl reference` times that oracle per step.

The timed form (`value`) is mixed precision with the learned row proposal,
whose network is first trained on the GPU (untimed) with the standard recipe
(leaves of the d = 128 and d = 1000 generators). Beside it: plain FP64 with
uniform sampling (`fp64_plain`, the reference point of the speedup) and the
two other precision x sampler arms. The oracle baseline compresses with the
uniform sampler (the network's weights come from the GPU path and are never
fed to the oracle).
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
COMMON = {"tol": 1e-6, "s0": 128, "s_max": 2048, "min_level": 2, "xi": 1.0, "sample_seed": 0}
WORKLOAD = dict(WORKLOADS["c2"], **COMMON)


def select_workload(name: str):
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


def build_inputs(torch, dev):
    from paper_1409_2802_gb300 import ffc
    rank, _, _ = _env_rank()
    P = workload_points(rank)
    Pd = torch.tensor(P, device=dev)
    tree = ffc.ffc_build_tree(Pd, WORKLOAD["leaf_size"])
    Pp = Pd[tree.perm].contiguous()
    return P, tree, Pp, workload_kernel(ffc, P)


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


def run_gpu_steps(torch, ffc, Pp, tree, k, precision, steps, warmup, flush_buf, stream, result=None, proposal=None,
                  qr_kw=None):
    W = WORKLOAD
    qr_kw = qr_kw or {}

    def step(res):
        return ffc.ffc_compress_tree(Pp, tree, k, tol=W["tol"], precision=precision, min_level=W["min_level"],
                                     s0=W["s0"], s_max=W["s_max"], xi=W["xi"], seed=W["sample_seed"], result=res,
                                     stream=stream, proposal=proposal, **qr_kw)

    res = result
    for _ in range(warmup):
        res = step(res)
    res.profile_enable(True)
    res.profile_reset()
    times = []
    for _ in range(steps):
        flush_buf.fill_(1.0)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        step(res)
        e1.record(stream)
        e1.synchronize()
        times.append(e0.elapsed_time(e1))
    prof = res.profile()
    res.profile_enable(False)
    return res, times, prof


def run_e2e(torch, ffc, P_host_perm, tree, k, precision, steps, warmup, stream, proposal=None, qr_kw=None):
    """Same metric through host buffers: pinned H2D inputs, compress, D2H results, every step."""
    W = WORKLOAD
    dev = P_host_perm.device if P_host_perm.is_cuda else torch.device("cuda")
    hP = P_host_perm.cpu().pin_memory()
    tree_host = {n: getattr(tree, n).cpu().pin_memory() for n in ("begin", "count", "centroid", "radius")}
    dP = torch.empty_like(hP, device=dev)
    dT = {n: torch.empty_like(v, device=dev) for n, v in tree_host.items()}
    dtree = ffc.DeviceTree(tree.depth, tree.perm, dT["begin"], dT["count"], dT["centroid"], dT["radius"])
    res = None
    h2d = hP.numel() * hP.element_size() + sum(v.numel() * v.element_size() for v in tree_host.values())
    d2h_bytes = []

    def step(res):
        with torch.cuda.stream(stream):
            dP.copy_(hP, non_blocking=True)
            for n in dT:
                dT[n].copy_(tree_host[n], non_blocking=True)
        res = ffc.ffc_compress_tree(dP, dtree, k, tol=W["tol"], precision=precision, min_level=W["min_level"],
                                    s0=W["s0"], s_max=W["s_max"], xi=W["xi"], seed=W["sample_seed"], result=res,
                                    stream=stream, proposal=proposal, **(qr_kw or {}))
        with torch.cuda.stream(stream):
            v = ffc.tree_result_views(res)
            out = {kk: v[kk].to("cpu", non_blocking=False) for kk in ("rank", "s", "status", "r22_rel", "skel", "T_off",
                                                                       "T")}
        d2h_bytes.append(sum(t.numel() * t.element_size() for t in out.values()))
        return res

    for _ in range(warmup):
        res = step(res)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        res = step(res)
    e1.record(stream)
    e1.synchronize()
    wall = time.perf_counter() - t0
    ms = e0.elapsed_time(e1)
    n_nodes = ffc.tree_result_views(res)["n_out"]
    return {"value": n_nodes * steps / (ms / 1e3), "unit": UNIT, "h2d_bytes_per_step": int(h2d),
            "d2h_bytes_per_step": int(statistics.mean(d2h_bytes[-steps:])), "wall_s": wall}


# --------------------------------------------------------------------------- oracle legs

def oracle_setup():
    from oracle import kernels as o_kernels
    from oracle import tree as o_tree
    P = workload_points()
    t = o_tree.build_tree(P, WORKLOAD["leaf_size"])
    return P[t.perm].astype("float64"), t, workload_kernel(o_kernels, P)


def oracle_nodes_in_order(t, seed=12345):
    import numpy as np
    nodes = np.array([i for i in range(t.n_nodes) if t.level[i] >= WORKLOAD["min_level"]])
    return list(np.random.default_rng(seed).permutation(nodes))


def oracle_compress(Pp, t, kernel, node):
    from oracle import compress as o_compress
    W = WORKLOAD
    return o_compress.compress_node(Pp, t, int(node), kernel, W["tol"], W["sample_seed"], W["s0"], W["s_max"],
                                    W["xi"])


_WORKER = {}


def _worker_init(name, barrier):
    """Pool worker: the oracle's inputs (points, tree, kernel), then wait for every other worker."""
    select_workload(name)
    _WORKER["state"] = oracle_setup()
    barrier.wait()


def _worker_compress(node):
    Pp, t, kernel = _WORKER["state"]
    oracle_compress(Pp, t, kernel, node)
    return int(node)


def cpu_leg(workers: int = 1) -> int:
    """Child process: compress nodes in a seeded random order, one JSON line per finished node.
    With workers > 1 the nodes go to a pool of single-threaded processes (spawned), each with its own
    copy of the oracle's inputs; the stream reports ready once every worker holds them."""
    if workers <= 1:
        Pp, t, kernel = oracle_setup()
        order = oracle_nodes_in_order(t)
        print(json.dumps({"ready": True, "of": len(order), "workers": 1}), flush=True)
        t0 = time.perf_counter()
        for i, node in enumerate(order):
            oracle_compress(Pp, t, kernel, node)
            print(json.dumps({"done": i + 1, "t": time.perf_counter() - t0}), flush=True)
        return 0
    import multiprocessing as mp
    from oracle import tree as o_tree
    P = workload_points()
    order = oracle_nodes_in_order(o_tree.build_tree(P, WORKLOAD["leaf_size"]))
    ctx = mp.get_context("spawn")
    with ctx.Manager() as mgr:
        barrier = mgr.Barrier(workers + 1)
        with ctx.Pool(workers, initializer=_worker_init, initargs=(WORKLOAD.get("name", "c2"), barrier)) as pool:
            barrier.wait()
            print(json.dumps({"ready": True, "of": len(order), "workers": workers}), flush=True)
            t0 = time.perf_counter()
            for i, _ in enumerate(pool.imap_unordered(_worker_compress, order, chunksize=1)):
                print(json.dumps({"done": i + 1, "t": time.perf_counter() - t0}), flush=True)
    return 0


class OracleStream:
    """The FP64 oracle compressing nodes in a seeded random order in a child process: one
    single-threaded process, or a pool of `workers` of them over the host cores.

    The child prints one line per finished node; the parent reads the count of
    finished nodes at any time. The nodes in progress when a window closes
    count as time spent, so a window's throughput is finished nodes / window.
    """

    def __init__(self, workers: int = 1):
        self.workers = max(1, int(workers))
        env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
        for k in ("RANK", "WORLD_SIZE", "LOCAL_RANK"):
            env.pop(k, None)
        self.proc = subprocess.Popen([sys.executable, os.path.abspath(__file__), "--_cpu-leg", str(self.workers),
                                      "--workload", WORKLOAD.get("name", "c2")], env=env,
                                     stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True,
                                     start_new_session=True)
        self.of, self.ready_t, self.done = None, None, 0
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            try:
                msg = json.loads(line)
            except ValueError:
                continue
            if msg.get("ready"):
                self.of = msg["of"]
                self.ready_t = time.perf_counter()
            elif "done" in msg:
                self.done = msg["done"]

    def wait_ready(self, timeout=900.0) -> bool:
        end = time.perf_counter() + timeout
        while self.ready_t is None and self.proc.poll() is None and time.perf_counter() < end:
            time.sleep(0.05)
        return self.ready_t is not None

    def window(self, seconds: float):
        """Sleep through one window; returns (nodes finished in it, its length)."""
        d0, t0 = self.done, time.perf_counter()
        end = t0 + seconds
        while self.proc.poll() is None and time.perf_counter() < end:
            time.sleep(0.05)
        return self.done - d0, time.perf_counter() - t0

    def close(self):
        # the child's own process group holds its pool workers
        try:
            os.killpg(self.proc.pid, 9)
        except (ProcessLookupError, PermissionError):
            self.proc.kill()
        self.proc.wait()


def finish_cpu_baseline(o: "OracleStream", min_seconds: float, when: str) -> dict:
    """Close an oracle stream after at least `min_seconds` of it; nodes finished / window."""
    try:
        if not o.wait_ready():
            return {"value": None, "unit": UNIT, "cores": o.workers, "kind": "oracle",
                    "sample": "oracle setup failed"}
        remaining = o.ready_t + min_seconds - time.perf_counter()
        if remaining > 0:
            o.window(remaining)
        el = time.perf_counter() - o.ready_t
        done = o.done
    finally:
        o.close()
    procs = "one thread" if o.workers == 1 else f"{o.workers} single-threaded processes, one node each at a time"
    return {"value": done / el, "unit": UNIT, "cores": o.workers, "kind": "oracle",
            "sample": (f"{done} of {o.of} nodes finished in a {el:.1f} s window (seeded random node order; the "
                       f"nodes still running at the end count as time spent), uniform sampler, {procs} "
                       f"(OMP/OpenBLAS = 1), {when}")}


def host_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def reference_arm(args, rank, world):
    """--impl reference: the FP64 CPU oracle; each step is one fixed time window of its node stream."""
    if rank != 0:
        return 0
    win = min(20.0, max(2.0, 150.0 / (args.steps + args.warmup)))
    o = OracleStream(args.cpu_workers or host_cores())
    try:
        if not o.wait_ready():
            print(json.dumps({"impl": "reference", "unavailable": "oracle setup failed"}))
            return 0
        for _ in range(args.warmup):
            o.window(win)
        done, el = 0, 0.0
        for _ in range(args.steps):
            dn, t = o.window(win)
            done += dn
            el += t
    finally:
        o.close()
    value = done / el
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 0, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": el * 1e3 / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD["workload"], "step": f"{win:.1f} s window of the oracle's node stream",
                   "l2": "n/a (CPU)"},
        "cpu_baseline": {"value": value, "unit": UNIT, "kind": "oracle", "cores": o.workers,
                         "sample": f"{done} nodes finished over {args.steps} windows of {win:.1f} s "
                                   f"(seeded random node order), {o.workers} single-threaded processes"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


FP32_PEAK_TFLOPS = 80.5   # 152 SMs x 128 FP32 lanes x 2 flops x 2.07 GHz (nominal)



def qr_traffic(precision_name, sampler, shape=None):
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
        if (rec.get("cpqr_sha256") == h and rec.get("workload") == WORKLOAD["workload"]
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
        return {"kernel": "eval_tc_kernel (split-BF16 mma.sync, FP32 accumulate)", "bound": "tensor",
                "achieved": tflops, "peak": peak, "unit": "TFLOP/s", "frac": tflops / peak,
                "tensor_work_tflops": 6.0 * tflops, "tensor_work_frac": 6.0 * tflops / peak,
                "peak_source": f"{peak_src} dense BF16, sustained (MEASURED_PEAKS.json bf16_tflops_sustained, "
                               "tcgen05 cuBLAS)",
                "gemm_flops_per_step": gemm, "ms_per_step": ms}
    peak = FP32_PEAK_TFLOPS if precision_name == "mixed" else FP64_PEAK_TFLOPS
    return {"kernel": "eval_kernel (SIMT)", "bound": "alu", "achieved": tflops, "peak": peak, "unit": "TFLOP/s",
            "frac": tflops / peak, "gemm_flops_per_step": gemm, "ms_per_step": ms,
            "peak_source": "nominal FP32 rate of GB300" if precision_name == "mixed" else "nominal FP64 rate of GB300"}


def qr_roofline(prof, steps, precision_name, peaks, peak_src, sampler="learned", shape=None):
    """Roofline of the pivoted QR from the library's live per-phase CUDA-event timing.

    Algorithmic bytes: one read and one write of every sampled block K' (s x n)
    per QR launch. The unblocked Householder QR streams the trailing matrix
    once per step, (s - k)(n - k) elements read and written at step k; that
    volume is reported as `streamed_gbs`, and the FP32/FP64 ALU rate beside it.
    """
    phase_ms = prof["ms"]
    qr_ms = phase_ms["qr"] / max(steps, 1)
    esz = 8.0 if precision_name == "fp64" else 4.0
    tflops = prof["qr_flops"] / steps / (qr_ms / 1e3) / 1e12 if qr_ms > 0 else 0.0
    gbs = prof["qr_bytes"] / steps / (qr_ms / 1e3) / 1e9 if qr_ms > 0 else 0.0
    streamed = prof["qr_flops"] / 2.0 * esz / steps / (qr_ms / 1e3) / 1e9 if qr_ms > 0 else 0.0
    hbm = peaks.get("hbm_gbs", 6775.3)
    if precision_name == "fp64":
        alu_peak, kern, src = FP64_PEAK_TFLOPS, "cpqr_kernel<double> (pivoted QR, FP64)", "nominal FP64 rate of GB300"
    else:
        alu_peak, kern, src = FP32_PEAK_TFLOPS, "cpqr_kernel<float> (pivoted QR, FP32 updates, FP64 norms)", \
            "nominal FP32 rate of GB300 (152 SMs x 128 lanes x 2.07 GHz)"
    traffic, traffic_src = qr_traffic(precision_name, sampler, shape)
    return {
        "kernel": kern, "bound": "hbm", "achieved": gbs, "peak": hbm, "unit": "GB/s", "frac": gbs / hbm,
        "traffic": traffic, "traffic_unit": "bytes per step (all QR launches of one call)",
        "traffic_source": traffic_src,
        "peak_source": f"{peak_src} HBM copy bandwidth (MEASURED_PEAKS.json hbm_gbs)",
        "streamed_gbs": streamed, "streamed_frac": streamed / hbm,
        "alu": {"achieved": tflops, "peak": alu_peak, "unit": "TFLOP/s", "frac": tflops / alu_peak, "source": src},
        "dominant_phase": max(phase_ms, key=phase_ms.get),
        "phase_ms_per_step": {k: v / steps for k, v in phase_ms.items()},
        "qr_ms_per_step_by_round": [round(v / steps, 3) for v in prof.get("qr_ms_round", [])],
        "nodes_per_step_by_round": [int(v // steps) for v in prof.get("items_round", [])],
        "qr_flops_per_step": prof["qr_flops"] / steps, "qr_bytes_per_step": prof["qr_bytes"] / steps,
        "eval": eval_roofline(prof, steps, precision_name, peaks, peak_src),
    }


def arm_errors(torch, ffc, Pp, tree, k, res, n_sample=12, seed=7):
    """Full-block ID error of a seeded sample of nodes of one arm's result (outside the timed region)."""
    import numpy as np
    W = WORKLOAD
    h = ffc.tree_result_to_host(res)
    v = ffc.tree_result_views(res)
    nodes = h["node"]
    pick = sorted(np.random.default_rng(seed).choice(len(nodes), min(n_sample, len(nodes)), replace=False).tolist())
    begin, count = tree.begin.cpu().numpy(), tree.count.cpu().numpy()
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
            "mean_s": float(h["s"].mean())}


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
                  "nodes_at_or_below_1e-5": int(np.sum(e <= 1e-5)), "mean_rank": a["mean_rank"],
                  "mean_s": a["mean_s"]}
    for samp in ("learned", "uniform"):
        a, b = f"mixed_{samp}", f"fp64_{samp}"
        if a in per_arm and b in per_arm:
            dmax = float(max(abs(x - y) for x, y in zip(per_arm[a]["errors"], per_arm[b]["errors"])))
            out[f"max_abs_diff_mixed_vs_fp64_{samp}"] = dmax
            out[f"within_1e-6_{samp}"] = dmax <= 1e-6
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="mixed", choices=["fp64", "mixed"],
                    help="precision of the timed form (value)")
    ap.add_argument("--sampler", default="learned", choices=["learned", "uniform"],
                    help="row sampler of the timed form; learned trains the proposal first (untimed)")
    ap.add_argument("--train-epochs", type=int, default=30)
    ap.add_argument("--train-nodes", type=int, default=100, help="training leaves per generator (d=128, d=1000)")
    ap.add_argument("--no-fp64-compare", action="store_true", help="skip the plain FP64 uniform arm and the others")
    ap.add_argument("--no-accuracy", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=30.0)
    ap.add_argument("--cpu-workers", type=int, default=0,
                    help="oracle processes for the all-cores CPU baseline and the reference arm (0 = every host core)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-autotune", action="store_true",
                    help="skip the QR launch-shape autotuner (untimed, before the timed form's steps)")
    ap.add_argument("--workload", default="c2", choices=sorted(WORKLOADS),
                    help="c2 (default, the headline): d=16 mixture; c3-laplace / c3-poly: d=128; c4: d=1000 FP32")
    ap.add_argument("--_cpu-leg", type=int, default=None, help=argparse.SUPPRESS)
    args = ap.parse_args()
    select_workload(args.workload)

    if args._cpu_leg is not None:
        return cpu_leg(args._cpu_leg)

    rank, world, local = _env_rank()
    oracle = OracleStream() if (rank == 0 and world == 1 and not args.no_cpu_baseline and args.impl == "ours") else None
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
    proposal, train_info = None, None
    if args.sampler == "learned":
        params, train_info = learned.train_standard(seed=0, epochs=args.train_epochs,
                                                    nodes_per_generator=args.train_nodes, device=dev)
        proj = torch.as_tensor(workloads.projections(WORKLOAD["d"], seed=7)).to(dev)
        proposal = (params, proj)
        torch.cuda.empty_cache()
    P, tree, Pp, kern = build_inputs(torch, dev)
    stream = torch.cuda.Stream(device=dev)
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    prec = precision_code(ffc, args.precision)
    peaks, peak_src = load_peaks()

    tuned = None
    if not args.no_autotune:
        from paper_1409_2802_gb300 import autotune
        W = WORKLOAD
        try:
            tuned = autotune.tune_tree(Pp, tree, kern, precision=prec, stream=stream, tol=W["tol"],
                                       min_level=W["min_level"], s0=W["s0"], s_max=W["s_max"], xi=W["xi"],
                                       seed=W["sample_seed"], proposal=proposal)
        except ffc.FFCError as e:             # the library's defaults then
            print(f"autotune skipped: {e}", file=sys.stderr)
            tuned = None
    qr_kw = {k_: tuned[k_] for k_ in ("qr_big_min_s", "qr_l2_budget_mb")} if tuned else {}

    def timed(prec_code, steps, warmup, prop, kw=None):
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()
        res, times, prof = run_gpu_steps(torch, ffc, Pp, tree, kern, prec_code, steps, warmup, flush, stream,
                                         proposal=prop, qr_kw=kw)
        torch.cuda.synchronize()
        total = max_over_ranks(sum(times), world, dev)
        if world > 1:
            torch.distributed.barrier()
        return res, total, prof

    clocks = ClockSampler(local)
    clocks.start()
    res, total_ms, prof = timed(prec, args.steps, args.warmup, proposal, qr_kw)
    clk = clocks.stop()
    n_nodes = int(ffc.tree_result_views(res)["n_out"])
    value = job_throughput(n_nodes, args.steps, world, total_ms)
    arm = f"{args.precision}_{args.sampler}"
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64" if prec == ffc.FP64 else "f32+f64", "data": "synthetic",
        "config": {"workload": WORKLOAD["workload"], "precision": args.precision, "sampler": args.sampler,
                   "nodes": n_nodes, "levels": f"2..{tree.depth}", "kernel": kernel_label(kern.h),
                   "points": WORKLOAD["points"], "tol": WORKLOAD["tol"],
                   "s": "128 doubling to 2048", "l2": "flushed between steps (512 MB write)",
                   "parallelism": f"replicas x{world}"},
        "clocks": clk, "gpu_launches": int(prof["launches"]),
        "roofline": qr_roofline(prof, args.steps, args.precision, peaks, peak_src, args.sampler, qr_kw or None),
    }
    if train_info is not None:
        line["config"]["proposal_training"] = train_info
    line["config"]["qr_launch_shape"] = (dict(tuned, source="autotune (timed form; other arms: defaults)")
                                         if tuned else {"source": "library defaults"})
    # each arm's sampled errors are taken as soon as it has run and its result is released, so
    # that only one arm's workspace is resident at a time
    errors = {}
    if not args.no_accuracy and rank == 0:
        errors[arm] = arm_errors(torch, ffc, Pp, tree, kern, res)
    res.close()
    del res
    if not args.no_fp64_compare:
        fsteps = max(3, args.steps // 3)
        arms = [("fp64", "uniform")]
        if args.sampler == "learned":
            arms += [("mixed", "uniform"), ("fp64", "learned")]
        other = {}
        for pname, sname in arms:
            key = f"{pname}_{sname}"
            if key == arm:
                continue
            r_, ms_, pf_ = timed(precision_code(ffc, pname), fsteps, 1, proposal if sname == "learned" else None)
            v_ = job_throughput(n_nodes, fsteps, world, ms_)
            other[key] = {"value": v_, "unit": UNIT, "ms_per_step": ms_ / fsteps, "steps": fsteps,
                          "roofline": qr_roofline(pf_, fsteps, pname, peaks, peak_src, sname)}
            if not args.no_accuracy and rank == 0:
                errors[key] = arm_errors(torch, ffc, Pp, tree, kern, r_)
            r_.close()
            del r_
        if "fp64_uniform" in other:
            line["fp64_plain"] = other.pop("fp64_uniform")
            line["speedup_vs_fp64"] = value / line["fp64_plain"]["value"]
        if other:
            line["arms"] = other
    if errors:
        line["accuracy"] = accuracy_summary(errors)
    if not args.no_e2e:
        line["e2e"] = run_e2e(torch, ffc, Pp, tree, kern, prec, max(3, args.steps // 2), 2, stream, proposal=proposal,
                              qr_kw=qr_kw)
    if oracle is not None:
        single = finish_cpu_baseline(oracle, args.cpu_seconds, "on a host core while the GPU steps ran")
        # every host core, after the GPU work (so that it does not compete with the GPU process's host thread)
        try:
            multi = finish_cpu_baseline(OracleStream(args.cpu_workers or host_cores()),
                                        min(20.0, args.cpu_seconds), "on the host cores after the GPU work")
        except (OSError, RuntimeError) as e:
            multi = {"value": None, "sample": f"all-cores oracle failed: {e}"}
        # a window in which no node finished (large blocks) says nothing: keep the longer single-core one
        line["cpu_baseline"] = multi if multi.get("value") else single
        line["cpu_baseline_single_core"] = single
    if rank == 0:
        print(json.dumps(line))
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
