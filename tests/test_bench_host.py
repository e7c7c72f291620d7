"""Host-side pieces of the benchmark on CPU: the reference arm's JSON line (the
FP64 oracle timed on the host cores), the QR traffic record and the rooflines."""
import json
import os
import subprocess
import sys

import bench

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_the_contract_line():
    """The oracle over a pool of two processes (the arm's default is every host core)."""
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "2",
                          "--warmup", "1", "--cpu-workers", "2", "--workload", "c2"], capture_output=True, text=True,
                         timeout=600, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    line = json.loads(out.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference"
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in line, key
    assert line["metric"] == bench.METRIC and line["unit"] == "nodes/s" and line["higher_is_better"] is True
    assert line["value"] > 0 and line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] >= 1
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["d2h_bytes_per_step"] == 0
    assert line["config"]["workload"] == bench.CONFIGS["c2"]["workload"]
    assert line["cpu_baseline"]["cores"] == 2
    # each step is one complete pass over the same fixed sample
    assert line["cpu_baseline"]["sample"].startswith("16 nodes (16 of c2)")


def test_traffic_record_applies_only_to_its_kernel_source_and_workload(tmp_path, monkeypatch):
    bench.select_workload("c2")
    t, src = bench.qr_traffic("mixed", "learned")
    if t is not None:                         # the committed record matches the current source
        assert t > 0 and src.startswith("profiles/")
    assert bench.qr_traffic("fp64", "uniform") == (None, None)
    bench.select_workload("c4")
    assert bench.qr_traffic("mixed", "learned") == (None, None)
    bench.select_workload("c2")
    # a record for another kernel source is ignored
    fake = tmp_path / "profiles"
    fake.mkdir()
    (fake / "cpqr_traffic_x.md").write_text("traffic_bytes_per_step: 5\ncpqr_sha256: 00\n"
                                            f"workload: {bench.WORKLOAD['workload']}\nprecision: mixed\n"
                                            "sampler: learned\n")
    csrc = tmp_path / "paper_1409_2802_gb300" / "csrc"
    csrc.mkdir(parents=True)
    (csrc / "cpqr.cu").write_text("// another source\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.qr_traffic("mixed", "learned") == (None, None)


def test_eval_roofline_bound_by_path():
    prof = {"ms": {"eval": 30.0}, "eval_flops": 3.0 * 1e12}
    bench.select_workload("c4")
    r = bench.eval_roofline(prof, 1, "mixed", {"bf16_tflops_sustained": 1710.8}, "measured")
    assert r["bound"] == "tensor" and abs(r["achieved"] - 2e12 / 0.030 / 1e12) < 1e-9
    assert abs(r["tensor_work_tflops"] - 6 * r["achieved"]) < 1e-9 and r["peak"] == 1710.8
    bench.select_workload("c2")                       # d = 16: the SIMT path
    r = bench.eval_roofline(prof, 1, "mixed", {}, "measured")
    assert r["bound"] == "alu" and r["peak"] == bench.FP32_PEAK_TFLOPS
    bench.select_workload("c3-laplace")               # Laplace stays SIMT at any d
    assert bench.eval_roofline(prof, 1, "mixed", {}, "measured")["bound"] == "alu"
    bench.select_workload("c2")


def test_oracle_sample_and_cpu_baseline_pool():
    """The oracle legs' node sample (the two deepest levels, fixed by the seed) and the all-cores CPU
    baseline: complete passes over it by a pool of single-threaded oracle processes."""
    items = bench.oracle_sample("c3")
    assert [p for p, _ in items] == ["c3-laplace"] * 16 + ["c3-poly"] * 16
    assert all(510 <= nd <= 2046 for _, nd in items)                  # levels 9 and 10 of the depth-10 tree
    assert items == bench.oracle_sample("c3")
    cb = bench.cpu_baseline_leg("c2", 2, 0.5)
    assert cb["cores"] == 2 and cb["kind"] == "oracle" and cb["value"] > 0 and "1 passes" in cb["sample"]


def test_combined_profiles_and_measured_alu_peaks():
    p1 = {"ms": {"sample": 1.0, "eval": 2.0, "qr": 3.0, "trsm": 4.0, "bookkeeping": 0.5}, "launches": 10,
          "qr_launches": 2, "qr_flops": 1e9, "eval_flops": 2e9, "qr_bytes": 3e9, "qr_ms_round": [1.0] * 8,
          "items_round": [2] * 8}
    c = bench.combine_profiles([p1, p1])
    assert c["ms"]["qr"] == 6.0 and c["launches"] == 20 and c["qr_bytes"] == 6e9 and c["items_round"][0] == 4
    r = bench.qr_roofline(c, 2, "mixed", {"hbm_gbs": 6000.0, "fp32_tflops": 60.0, "fp32_tflops_how": "probe"},
                          "measured")
    assert abs(r["achieved"] - 3e9 / (3.0 / 1e3) / 1e9) < 1e-9 and r["alu"]["peak"] == 60.0
    assert r["alu"]["source"].startswith("measured") and r["peak"] == 6000.0
    assert bench.qr_roofline(c, 2, "fp64", {}, "measured")["alu"]["peak"] == bench.FP64_PEAK_TFLOPS


def test_autotuner_search_order_and_fallback(monkeypatch):
    """The tuner's coordinate search with the timing mocked: the threshold first (at 96 MB), then the
    budget at the best threshold; a candidate that fails is recorded and skipped."""
    import pytest
    torch = pytest.importorskip("torch")
    from paper_1409_2802_gb300 import autotune, ffc
    cost = {(512, 96): 5.0, (1024, 96): 3.0, (2048, 96): 4.0, (1 << 30, 96): 9.0, (1024, 64): 3.5,
            (1024, 128): 2.5}
    calls = []

    def fake(points_perm, tree, kernel, stream, reps, precision, qr_big_min_s, qr_l2_budget_mb, **kw):
        calls.append((qr_big_min_s, qr_l2_budget_mb))
        if (qr_big_min_s, qr_l2_budget_mb) == (2048, 96):
            raise ffc.FFCError(ffc.FFC_E_NOMEM, "out of memory")
        return cost.get((qr_big_min_s, qr_l2_budget_mb), 6.0)

    monkeypatch.setattr(autotune, "_time_call", fake)
    best = autotune.tune_tree(None, None, None, precision=ffc.MIXED, stream=object())
    assert calls == [(512, 96), (1024, 96), (2048, 96), (1 << 30, 96), (1024, 64), (1024, 128)]
    assert (best["qr_big_min_s"], best["qr_l2_budget_mb"], best["ms"]) == (1024, 128, 2.5)
    assert any("error" in row for row in best["table"])
    calls.clear()
    best = autotune.tune_tree(None, None, None, precision=ffc.FP64, stream=object())
    assert calls == [(1 << 30, 96), (1 << 30, 64), (1 << 30, 128)]
