"""GPU test of ffc_id_noalloc, the allocation-free variant of ffc_id.

Some callers cannot allocate device memory at the moment they call the
library: the device memory may already be owned by a framework's caching
allocator, a latency-critical loop may not tolerate an allocation's implicit
synchronisation, or the memory budget may be fixed up front. For them
ffc_id_noalloc keeps its scratch in one fixed device array. This test calls
it through the C ABI and checks that it returns what ffc_id returns (same
rank, skeleton, residual, and interpolation matrix to the parity tolerance),
on two calls in a row: the second call starts from whatever the first left in
the shared array.
"""
import ctypes

import numpy as np
import pytest
import torch

import workloads

pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_1409_2802_gb300 import ffc  # noqa: E402

DEV = torch.device("cuda:0")


def _run(entry, K, r_max, tol):
    """Call ffc_id or ffc_id_noalloc directly through the C ABI on a copy of K (s x n)."""
    s, n = K.shape
    Kst = torch.tensor(np.ascontiguousarray(K.T), device=DEV)      # column-major s x n, ld = s
    ldt = max(int(r_max), 1)
    skel = torch.full((n,), -1, dtype=torch.int32, device=DEV)
    T = torch.zeros((n, ldt), dtype=torch.float64, device=DEV)
    rank, r22 = ctypes.c_int64(-1), ctypes.c_double(-1.0)
    st = getattr(ffc.lib(), entry)(ctypes.c_void_p(Kst.data_ptr()), s, n, s, ffc.FP64, int(r_max), float(tol),
                                   ctypes.c_void_p(skel.data_ptr()), ctypes.c_void_p(T.data_ptr()), ldt,
                                   ctypes.byref(rank), ctypes.byref(r22),
                                   ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    r = rank.value
    return st, r, r22.value, skel.cpu().numpy(), T[: n - r, :r].t().cpu().numpy()


def _problems():
    X, Y = workloads.single_block(0)
    g = np.random.default_rng(0)
    rows = g.choice(Y.shape[0], 256, replace=False)
    D2 = ((Y[rows][:, None, :] - X[None, :, :]) ** 2).sum(-1)
    gauss = np.exp(-D2 / 2.0)                                       # Gaussian kernel block, h = 1
    rand = workloads.random_matrix(300, 1000, seed=4, decay=0.9)
    return [(gauss, 64, 0.0), (rand, 150, 1e-9)]


def _same(a, b, K):
    st_a, r_a, r22_a, skel_a, T_a = a
    st_b, r_b, r22_b, skel_b, T_b = b
    assert st_a == st_b
    assert r_a == r_b
    assert abs(r22_a - r22_b) <= 1e-10
    assert np.array_equal(skel_a, skel_b)
    # the reconstructions K(:,J) P agree to rounding
    J = skel_a[:r_a]
    diff = np.linalg.norm(K[:, J] @ (T_a - T_b)) / np.linalg.norm(K)
    assert diff <= 1e-12, diff


def test_noalloc_matches_ffc_id_on_two_calls_in_a_row():
    probs = _problems()
    ref = [_run("ffc_id", K, r, tol) for K, r, tol in probs]
    first = [_run("ffc_id_noalloc", K, r, tol) for K, r, tol in probs]       # call 1, call 2
    second = [_run("ffc_id_noalloc", K, r, tol) for K, r, tol in probs]      # again, reusing the array
    for (K, _, _), a, b, c in zip(probs, ref, first, second):
        _same(a, b, K)
        _same(a, c, K)
    assert first[0][1] == 64 and first[0][0] == ffc.FFC_OK


def test_noalloc_at_its_stated_limits():
    """The largest problem the fixed scratch holds, n = FFC_NOALLOC_MAX_COLS columns, rank cap
    FFC_NOALLOC_MAX_RANK and s = 2048 rows (every region of the scratch at its full size), and the
    same width with a single row, against ffc_id, twice in a row."""
    n, r_max = 16384, 256
    K = workloads.random_matrix(2048, n, seed=12, decay=0.97)
    ref = _run("ffc_id", K, r_max, 0.0)
    assert ref[1] == r_max
    for _ in range(2):
        _same(ref, _run("ffc_id_noalloc", K, r_max, 0.0), K)
    K1 = workloads.random_matrix(1, n, seed=13)
    ref1 = _run("ffc_id", K1, 4, 0.0)
    assert ref1[1] == 1
    for _ in range(2):
        _same(ref1, _run("ffc_id_noalloc", K1, 4, 0.0), K1)


def test_noalloc_rejects_sizes_beyond_its_scratch():
    rank, r22 = ctypes.c_int64(0), ctypes.c_double(0.0)
    n = 16385                                                        # one column past FFC_NOALLOC_MAX_COLS
    st = ffc.lib().ffc_id_noalloc(None, 8, n, 8, ffc.FP64, 4, 0.0, None, None, 4, ctypes.byref(rank),
                                  ctypes.byref(r22), None)
    assert st == ffc.FFC_E_INVALID
    assert b"16384" in ffc.lib().ffc_last_error()
    st = ffc.lib().ffc_id_noalloc(None, 512, 1000, 512, ffc.FP64, 300, 0.0, None, None, 300, ctypes.byref(rank),
                                  ctypes.byref(r22), None)
    assert st == ffc.FFC_E_INVALID                                   # rank cap 300 > 256
