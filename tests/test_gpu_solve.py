"""GPU test of the mixed-precision triangular solve (ffc_params.solve): T = R11^-1 R12 by FP32 solves
refined once (the default) against the FP64 back-substitution, on the same QR.

What can be compared. The mixed path's R comes from an FP32 QR, so T is only determined by that data to
about cond(R11) 2^-24 whichever precision solves it; what reaches the ID is the residual R11 T - R12
(on the sampled block, K'(:, J) (T_a - T_b) = Q R11 (T_a - T_b)). One step of refinement with an exact
residual leaves a residual of about cond(R11) 2^-48 ||R11|| ||T||, far below the FP32 data's own error,
so:
* ranks, skeletons, samples and statuses are identical (the QR is the same);
* on the sampled block, ||K'(:, J) (T_default - T_fp64)||_F <= 1e-7 ||K'||_F;
* the full-block errors (FP64, streamed) agree to 1e-7, ten times below reading R2's 1e-6.
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


def _case(kind):
    if kind == "gaussian":
        P = workloads.gaussian_mixture(N=16384, d=16, k=8, seed=21)
        k = ffc.Kernel(ffc.GAUSSIAN, h=2.0)
    else:
        P = workloads.gaussian_mixture(N=16384, d=16, k=8, seed=22)
        k = ffc.Kernel(ffc.POLYNOMIAL, h=16.0, c=1.0, p=3)
    t = ffc.ffc_build_tree(torch.tensor(P, device=DEV), 256)
    Pp = torch.tensor(P, device=DEV)[t.perm].contiguous()
    return Pp, t, k


def _T(out, i, n):
    r = int(out["rank"][i])
    T = out["T"][out["T_off"][i]: out["T_off"][i] + r * (n - r)].reshape(n - r, r).T
    skel = out["skel"][out["skel_off"][i]: out["skel_off"][i] + n].astype(np.int64)
    return skel, T, r


@pytest.mark.parametrize("kind", ["gaussian", "cubic"])
def test_refined_solve_matches_the_fp64_solve_through_the_residual(kind):
    Pp, t, k = _case(kind)
    kw = dict(tol=1e-6, precision=ffc.MIXED, s0=128, s_max=2048)
    a = ffc.tree_result_to_host(ffc.ffc_compress_tree(Pp, t, k, solve=ffc.SOLVE_DEFAULT, **kw))
    b = ffc.tree_result_to_host(ffc.ffc_compress_tree(Pp, t, k, solve=ffc.SOLVE_FP64, **kw))
    for key in ("node", "rank", "s", "status", "rows", "skel"):
        assert np.array_equal(a[key], b[key]), key
    count, begin = t.count.cpu().numpy(), t.begin.cpu().numpy()
    big = np.flatnonzero(a["rank"] >= 32)
    assert big.size > 0
    for i in big[np.linspace(0, big.size - 1, min(10, big.size)).astype(int)]:
        node = int(a["node"][i])
        b0, n = int(begin[node]), int(count[node])
        if n > 4096:
            continue
        skel, Ta, r = _T(a, i, n)
        _, Tb, _ = _T(b, i, n)
        rows = torch.tensor(a["rows"][a["rows_off"][i]: a["rows_off"][i] + a["s"][i]], device=DEV)
        X = Pp[b0: b0 + n]
        K, _ = ffc.ffc_eval_block(k, Pp, rows, X, precision=ffc.FP64)
        K = K.cpu().numpy()
        res = np.linalg.norm(K[:, skel[:r]] @ (Ta - Tb)) / np.linalg.norm(K)
        assert res <= 1e-7, (node, r, res)
        far = ffc.ffc_far_field(Pp, x_c=t.centroid[node], radius=float(t.radius[node]), ex_begin=b0, ex_end=b0 + n)
        Y = Pp[far][:16384].contiguous()
        sk = torch.tensor(skel, device=DEV, dtype=torch.int32)
        e_a = ffc.ffc_id_error(k, Y, X, sk, torch.tensor(Ta, device=DEV), r)
        e_b = ffc.ffc_id_error(k, Y, X, sk, torch.tensor(Tb, device=DEV), r)
        assert abs(e_a - e_b) <= 1e-7, (node, e_a, e_b)
