"""GPU test of the library's bounded device waits (failure detection without a fault).

The pivoted QR of a block with several CTAs per block synchronises them once
per step through a barrier in global memory that polls a bounded number of
times. With the limit set to zero, a barrier that is not already complete
gives up at once: the QR stops, the call reports FFC_E_TIMEOUT, and the device
stays usable, so the same problem then factors correctly with the default
limit restored. Nothing here faults, traps or hangs the GPU: the wait that
runs out is an ordinary polling loop that returns.
"""
import numpy as np
import pytest
import torch

import workloads

pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_1409_2802_gb300 import ffc  # noqa: E402

DEV = torch.device("cuda:0")


def _block():
    # s = 256 rows, n = 2048 columns: the QR runs it on a group of many CTAs
    return workloads.random_matrix(256, 2048, seed=21, decay=0.97)


def test_qr_wait_that_runs_out_returns_timeout_and_the_device_recovers():
    K = _block()
    ref = ffc.ffc_id(torch.tensor(K.T.copy(), device=DEV), 64, 0.0)
    try:
        ffc.ffc_set_wait_limit(0)
        with pytest.raises(ffc.FFCError) as e:
            ffc.ffc_id(torch.tensor(K.T.copy(), device=DEV), 64, 0.0)
        assert e.value.status == ffc.FFC_E_TIMEOUT
        assert "timed out" in ffc.lib().ffc_last_error().decode()
    finally:
        ffc.ffc_set_wait_limit(-1)
    torch.cuda.synchronize()                       # the context is intact
    again = ffc.ffc_id(torch.tensor(K.T.copy(), device=DEV), 64, 0.0)
    assert again[2] == ref[2] == 64 and again[4] == ffc.FFC_OK
    assert torch.equal(again[0], ref[0]) and torch.equal(again[1], ref[1])


def test_tree_nodes_report_timeout_and_the_next_call_is_clean():
    P = workloads.gaussian_mixture(N=8192, d=8, k=4, seed=22)
    tree = ffc.ffc_build_tree(torch.tensor(P, device=DEV), 256)
    Pp = torch.tensor(P, device=DEV)[tree.perm].contiguous()
    k = ffc.Kernel(ffc.GAUSSIAN, h=1.5)
    clean = ffc.tree_result_to_host(ffc.ffc_compress_tree(Pp, tree, k, tol=1e-6, s0=64, s_max=1024))
    try:
        ffc.ffc_set_wait_limit(0)
        out = ffc.tree_result_to_host(ffc.ffc_compress_tree(Pp, tree, k, tol=1e-6, s0=64, s_max=1024))
    finally:
        ffc.ffc_set_wait_limit(-1)
    st = out["status"]
    # the large nodes run on groups of CTAs and time out; a node that one CTA factors has no wait
    assert np.any(st == ffc.FFC_E_TIMEOUT)
    assert np.all((st == ffc.FFC_E_TIMEOUT) | (st == clean["status"]))
    after = ffc.tree_result_to_host(ffc.ffc_compress_tree(Pp, tree, k, tol=1e-6, s0=64, s_max=1024))
    for key in ("status", "rank", "s", "skel", "T"):
        assert np.array_equal(after[key], clean[key]), key
