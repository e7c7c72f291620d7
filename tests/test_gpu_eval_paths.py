"""GPU parity of the evaluation paths of the mixed-precision Gaussian and polynomial blocks against the
FP64 oracle (oracle/kernels.kernel_block): the tcgen05 path (TMA-staged BF16 planes, TMEM
accumulators; each of its tile variants, 128 x 256 and 128 x 128 tiles with 32-, 64- and 128-byte
swizzled stages) and the mma.sync path (128 x 128 tiles) compute the same split-BF16
products in different summation orders, so both are held to the FP32 rounding bound of the
tensor-core test in test_gpu_mixed.py, on ragged shapes spanning several tiles, d not a multiple of
the 32-coordinate stage, FP32 and FP64 points. The tree compression with either path reaches the same
ranks and errors, and a bounded wait of the tcgen05 pipeline that runs out reports FFC_E_TIMEOUT with
the device still usable.
"""
import numpy as np
import pytest
import torch

import workloads
from oracle import kernels as o_kernels

pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_1409_2802_gb300 import ffc  # noqa: E402

DEV = torch.device("cuda:0")
U = 2.0 ** -24


def cu(a):
    return torch.tensor(np.ascontiguousarray(a), device=DEV)


def _bound(kind, Y64, X64, centre, h, Ko, d):
    # the FP32 rounding bound of D2 (Gaussian) or of the inner product (polynomial), as in test_gpu_mixed
    if kind == o_kernels.GAUSSIAN:
        yn = np.sum((Y64 - centre) ** 2, axis=1)
        xn = np.sum((X64 - centre) ** 2, axis=1)
        return Ko * ((d + 16) * 4 * U * (yn[:, None] + xn[None, :]) / (2 * h * h) + 4 * U) + 1e-30
    dots = np.abs(Y64) @ np.abs(X64).T
    base = Y64 @ X64.T / h + 1.0
    return 3 * np.abs(base) ** 2 * ((d + 16) * 4 * U * dots / h + 4 * U * np.abs(base)) + 1e-30


def _case(kind, d, s, n, pts, seed):
    g = np.random.default_rng(seed)
    X = g.standard_normal((n, d)) / np.sqrt(d)
    Y = g.standard_normal((s + 200, d)) / np.sqrt(d) + 0.4 / np.sqrt(d)
    Y[:30] = X[:30] + 1e-3 * g.standard_normal((30, d)) / np.sqrt(d)    # near-coincident pairs (D2 cancels)
    if pts == "f32":
        X, Y = X.astype(np.float32), Y.astype(np.float32)
    rows = np.concatenate([np.arange(30), g.choice(np.arange(30, s + 200), s - 30, replace=False)]).astype(np.int64)
    return X, Y, rows


def _eval(path, kind, X, Y, rows, h, centre):
    ffc.ffc_set_eval_path(path)
    try:
        Kg, _ = ffc.ffc_eval_block(ffc.Kernel(kind, h=h), cu(Y), cu(rows), cu(X), precision=ffc.MIXED,
                                   center=cu(centre))
    finally:
        ffc.ffc_set_eval_path(ffc.EVAL_DEFAULT)
    return Kg.double().cpu().numpy()


PATHS = [ffc.EVAL_TCGEN05, ffc.EVAL_MMA_SYNC] + [ffc.EVAL_TCGEN05_TILE0 + v for v in range(ffc.EVAL_TCGEN05_TILES)]


@pytest.mark.parametrize("path", PATHS)
@pytest.mark.parametrize("kind,d,s,n,pts", [
    (o_kernels.GAUSSIAN, 64, 300, 777, "f64"),
    (o_kernels.GAUSSIAN, 100, 1000, 3000, "f64"),     # d off the stage width; 8 x 12 tiles, ragged both ways
    (o_kernels.GAUSSIAN, 1000, 257, 513, "f32"),      # one row past a tile, one column past two
    (o_kernels.POLYNOMIAL, 128, 300, 777, "f64"),
    (o_kernels.POLYNOMIAL, 33, 129, 2049, "f32"),
])
def test_eval_path_matches_oracle(path, kind, d, s, n, pts):
    X, Y, rows = _case(kind, d, s, n, pts, seed=d + s)
    h = 0.8 if kind == o_kernels.GAUSSIAN else 1.0 / d
    X64, Y64 = X.astype(np.float64), Y.astype(np.float64)
    Ko, _ = o_kernels.kernel_block(o_kernels.Kernel(kind, h=h), Y64[rows], X64)
    centre = X64.mean(axis=0)
    Kg = _eval(path, kind, X, Y, rows, h, centre)
    assert Kg.shape == Ko.shape
    bound = _bound(kind, Y64[rows], X64, centre, h, Ko, d)
    assert np.all(np.abs(Kg - Ko) <= bound), float(np.max(np.abs(Kg - Ko) / bound))


def test_tcgen05_and_mma_sync_paths_agree():
    """Same planes, same six products: the two tensor-core paths differ by FP32 summation order only."""
    X, Y, rows = _case(o_kernels.GAUSSIAN, 256, 512, 1024, "f64", seed=5)
    centre = X.mean(axis=0)
    a = _eval(ffc.EVAL_TCGEN05, o_kernels.GAUSSIAN, X, Y, rows, 1.0, centre)
    b = _eval(ffc.EVAL_MMA_SYNC, o_kernels.GAUSSIAN, X, Y, rows, 1.0, centre)
    assert np.max(np.abs(a - b)) <= 1e-5 * np.max(np.abs(b))


def test_default_path_is_tcgen05_above_64_coordinates():
    X, Y, rows = _case(o_kernels.POLYNOMIAL, 96, 200, 300, "f32", seed=9)
    dflt = _eval(ffc.EVAL_DEFAULT, o_kernels.POLYNOMIAL, X, Y, rows, 1.0 / 96, X.mean(axis=0))
    t5 = _eval(ffc.EVAL_TCGEN05, o_kernels.POLYNOMIAL, X, Y, rows, 1.0 / 96, X.mean(axis=0))
    assert np.array_equal(dflt, t5)


def test_tree_compression_with_either_tensor_path():
    """d = 128 Gaussian mixture, mixed precision: the tree reaches the same statuses and (up to a rank
    step at a rounding-level pivot) the same ranks with both paths."""
    P = workloads.gaussian_mixture(N=16384, d=128, k=4, seed=6)
    t = ffc.ffc_build_tree(cu(P), 256)
    Pp = cu(P)[t.perm].contiguous()
    k = ffc.Kernel(ffc.GAUSSIAN, h=3.0)
    outs = {}
    for path in (ffc.EVAL_TCGEN05, ffc.EVAL_MMA_SYNC):
        outs[path] = ffc.tree_result_to_host(ffc.ffc_compress_tree(Pp, t, k, tol=1e-5, precision=ffc.MIXED, s0=128,
                                                                   s_max=1024, eval_path=path))
    a, b = outs[ffc.EVAL_TCGEN05], outs[ffc.EVAL_MMA_SYNC]
    assert np.array_equal(a["node"], b["node"]) and np.array_equal(a["s"], b["s"])
    assert np.array_equal(a["status"], b["status"])
    assert np.all(np.abs(a["rank"] - b["rank"]) <= 1)
    assert np.mean(a["rank"] == b["rank"]) >= 0.9
    ok = a["status"] == 0
    assert np.all(a["r22_rel"][ok] <= 1e-5) and np.all(b["r22_rel"][ok] <= 1e-5)


def test_tcgen05_wait_that_runs_out_returns_timeout_and_the_device_recovers():
    """With the poll limit at zero the epilogue's first wait for a 32-stage accumulator gives up: every
    role leaves its loop, the copies and products in flight drain, TMEM is freed, and the call
    reports FFC_E_TIMEOUT; the same block then evaluates correctly with the default limit."""
    X, Y, rows = _case(o_kernels.GAUSSIAN, 1000, 1024, 2048, "f32", seed=13)
    centre = X.astype(np.float64).mean(axis=0)
    ref = _eval(ffc.EVAL_TCGEN05, o_kernels.GAUSSIAN, X, Y, rows, 1.0, centre)
    ffc.ffc_set_eval_path(ffc.EVAL_TCGEN05)
    try:
        ffc.ffc_set_wait_limit(0)
        with pytest.raises(ffc.FFCError) as e:
            ffc.ffc_eval_block(ffc.Kernel(ffc.GAUSSIAN, h=1.0), cu(Y), cu(rows), cu(X), precision=ffc.MIXED,
                               center=cu(centre))
        assert e.value.status == ffc.FFC_E_TIMEOUT
    finally:
        ffc.ffc_set_wait_limit(-1)
        ffc.ffc_set_eval_path(ffc.EVAL_DEFAULT)
    torch.cuda.synchronize()
    again = _eval(ffc.EVAL_TCGEN05, o_kernels.GAUSSIAN, X, Y, rows, 1.0, centre)
    assert np.array_equal(again, ref)


def test_autotuner_picks_an_evaluation_path_per_bucket(tmp_path):
    from paper_1409_2802_gb300 import autotune
    k = ffc.Kernel(ffc.GAUSSIAN, h=2.0)
    cache = str(tmp_path / "eval_tune.json")
    a = autotune.tune_eval(k, 128, 3000, ffc.MIXED, s=512, cache_path=cache)
    assert a["source"] == "measured" and a["eval_path"] in autotune.EVAL_CANDIDATES
    assert set(a["table"]) == {str(p) for p in autotune.EVAL_CANDIDATES}
    b = autotune.tune_eval(k, 128, 4000, ffc.MIXED, s=512, cache_path=cache)    # same bucket (4096): cached
    assert b["source"] == "cache" and b["eval_path"] == a["eval_path"]
    assert autotune.tune_eval(ffc.Kernel(ffc.LAPLACE), 128, 3000)["eval_path"] == ffc.EVAL_DEFAULT
    P = workloads.gaussian_mixture(N=16384, d=64, k=4, seed=3)
    t = ffc.ffc_build_tree(cu(P), 256)
    Pp = cu(P)[t.perm].contiguous()
    tt = autotune.tune_tree_eval(Pp, t, k, ffc.MIXED, s_probe=256, cache_path=cache)
    assert tt["source"] == "measured" and tt["eval_path"] in autotune.EVAL_CANDIDATES
    assert set(tt["table"]) == {str(p) for p in autotune.EVAL_CANDIDATES}
    assert all(v > 0 for v in tt["table"].values())
    assert autotune.tune_tree_eval(Pp, t, k, ffc.MIXED, s_probe=256, cache_path=cache)["source"] == "cache"
