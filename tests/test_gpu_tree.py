"""GPU parity of the tree path: ffc_build_tree and ffc_compress_tree vs the oracle.

Small trees are compared node by node; at the benchmark's full size (N=65,536,
d=16, leaf 256, Gaussian h=2, tol 1e-6) every node is checked for the
properties that hold at any size and a seeded sample of nodes against the
oracle's per-node compression.
"""
import numpy as np
import pytest
import torch

import workloads
from oracle import compress as o_compress
from oracle import interp as o_interp
from oracle import kernels as o_kernels
from oracle import tree as o_tree
from parity import check_learned_node, far_rows_subset, fp64_error_ok, node_id

pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_1409_2802_gb300 import ffc  # noqa: E402

DEV = torch.device("cuda:0")


def cu(a):
    return torch.tensor(np.ascontiguousarray(a), device=DEV)


def _build_both(P, leaf):
    t_o = o_tree.build_tree(P, leaf)
    t_g = ffc.ffc_build_tree(cu(P), leaf)
    return t_o, t_g


@pytest.mark.parametrize("N,d,leaf", [(4096, 4, 256), (5000, 16, 300), (3001, 130, 100)])
def test_build_tree_matches_oracle(N, d, leaf):
    P = workloads.gaussian_mixture(N=N, d=d, k=4, seed=N)
    t_o, t_g = _build_both(P, leaf)
    assert t_g.depth == t_o.depth
    assert np.array_equal(t_g.perm.cpu().numpy(), t_o.perm)
    assert np.array_equal(t_g.begin.cpu().numpy(), t_o.begin)
    assert np.array_equal(t_g.count.cpu().numpy(), t_o.count)
    np.testing.assert_allclose(t_g.centroid.cpu().numpy(), t_o.centroid, rtol=0, atol=1e-12)
    np.testing.assert_allclose(t_g.radius.cpu().numpy(), t_o.radius, rtol=1e-13)


def _compare_nodes(out, t_o, Pp, kernel_o, tol, nodes, s0, s_max, seed=0, check_error=True, subset=False):
    index = {int(nd): i for i, nd in enumerate(out["node"])}
    for node in nodes:
        i = index[node]
        ref = o_compress.compress_node(Pp, t_o, node, kernel_o, tol, seed, s0, s_max)
        s = int(out["s"][i])
        assert s == ref.s, node
        rows = out["rows"][out["rows_off"][i]: out["rows_off"][i] + s]
        assert np.array_equal(rows, ref.rows), node
        assert int(out["far_count"][i]) in (-1, ref.far_count)
        assert int(out["status"][i]) == ref.status, node
        r = int(out["rank"][i])
        assert r == ref.rank, (node, r, ref.rank)
        assert abs(out["r22_rel"][i] - ref.r22_rel) <= 1e-10
        n = int(t_o.count[node])
        skel, T, r = node_id(out, i, n)
        P_g = o_interp.assemble_P(skel, T, n)
        assert np.array_equal(P_g[:, skel[:r]], np.eye(r))      # P contains I_r
        if check_error and r > 0:
            b = int(t_o.begin[node])
            if subset:
                far = far_rows_subset(Pp, t_o, node)
            else:
                from oracle.sampling import far_field_mask
                far = far_field_mask(Pp, t_o.centroid[node], t_o.radius[node], 1.0, b, b + n)
            e_g = o_interp.full_block_error(kernel_o, Pp[far], Pp[b:b + n], skel, T)
            e_o = o_interp.full_block_error(kernel_o, Pp[far], Pp[b:b + n], ref.skel_perm, ref.T)
            assert fp64_error_ok(e_g, e_o), (node, e_g, e_o, abs(e_g - e_o))
            # the two interpolation operators themselves: ||K'(:,J)(P_g - P_o)|| small against ||K'||
            Kn, _ = o_kernels.kernel_block(kernel_o, Pp[rows], Pp[b:b + n])
            P_o = o_interp.assemble_P(ref.skel_perm, ref.T, n)
            if np.array_equal(skel[:r], ref.skel_perm[:r]):
                dP = np.linalg.norm(Kn[:, skel[:r]] @ (P_g - P_o)) / np.linalg.norm(Kn)
                assert dP <= 1e-12, (node, dP)


def test_compress_small_tree_every_node():
    P = workloads.gaussian_mixture(N=4096, d=4, k=4, seed=1)
    t_o, t_g = _build_both(P, 256)
    Pp = P[t_o.perm]
    ko = o_kernels.Kernel(o_kernels.GAUSSIAN, h=1.0)
    res = ffc.ffc_compress_tree(cu(Pp), t_g, ffc.Kernel(ffc.GAUSSIAN, h=1.0), tol=1e-6, s0=32, s_max=512)
    out = ffc.tree_result_to_host(res)
    nodes = [i for i in range(t_o.n_nodes) if t_o.level[i] >= 2]
    assert list(out["node"]) == nodes
    _compare_nodes(out, t_o, Pp, ko, 1e-6, nodes, 32, 512)
    # the result object is reusable: a second call gives identical outputs
    out2 = ffc.tree_result_to_host(ffc.ffc_compress_tree(cu(Pp), t_g, ffc.Kernel(ffc.GAUSSIAN, h=1.0), tol=1e-6,
                                                         s0=32, s_max=512, result=res))
    for key in ("rank", "s", "rows", "skel", "T", "r22_rel"):
        assert np.array_equal(out[key], out2[key]), key


def test_compress_laplace_and_polynomial_small():
    P = workloads.gaussian_mixture(N=3000, d=6, k=3, seed=2)
    t_o, t_g = _build_both(P, 200)
    Pp = P[t_o.perm]
    for kind, h in ((o_kernels.LAPLACE, 1.0), (o_kernels.POLYNOMIAL, 6.0)):
        ko = o_kernels.Kernel(kind, h=h)
        out = ffc.tree_result_to_host(ffc.ffc_compress_tree(cu(Pp), t_g, ffc.Kernel(kind, h=h), tol=1e-6, s0=32,
                                                            s_max=256))
        nodes = [i for i in range(t_o.n_nodes) if t_o.level[i] >= 2]
        _compare_nodes(out, t_o, Pp, ko, 1e-6, nodes[::3], 32, 256)


def test_compress_full_size_gaussian_d16():
    """Benchmark configuration: every node's invariants, 12 seeded nodes vs the oracle."""
    P = workloads.gaussian_mixture(N=65536, d=16, k=8, seed=0)
    t_o, t_g = _build_both(P, 256)
    Pp = P[t_o.perm]
    res = ffc.ffc_compress_tree(cu(Pp), t_g, ffc.Kernel(ffc.GAUSSIAN, h=2.0), tol=1e-6, s0=128, s_max=2048)
    out = ffc.tree_result_to_host(res)
    assert out["n_out"] == 508
    st = out["status"]
    assert np.all((st == 0) | (st == ffc.FFC_E_TOL_NOT_REACHED))
    ok = st == 0
    assert np.all(out["r22_rel"][ok] <= 1e-6)
    cap = np.minimum(np.where(out["s"] < 2 * out["s"], out["s"] // 2, out["s"]), t_o.count[out["node"]])
    assert np.all(out["rank"] <= np.maximum(cap, out["s"]))
    g = np.random.default_rng(0)
    nodes = sorted(g.choice(out["node"], 12, replace=False).tolist())
    # full-block errors on a far-field subset of about 4,096 rows per node, for both IDs
    _compare_nodes(out, t_o, Pp, o_kernels.Kernel(o_kernels.GAUSSIAN, h=2.0), 1e-6, nodes, 128, 2048,
                   subset=True)


def test_compress_tree_learned_sampler_matches_oracle():
    """Learned sampler, FP64, every node: the drawn rows are the oracle's best keys up to the
    rounding of the FP32 logits, and the ID on those rows is the oracle's."""
    P = workloads.gaussian_mixture(N=4096, d=4, k=4, seed=3)
    t_o, t_g = _build_both(P, 256)
    Pp = P[t_o.perm]
    ko = o_kernels.Kernel(o_kernels.GAUSSIAN, h=1.0)
    g = np.random.default_rng(1)
    theta = (workloads.mlp_init(4).astype(np.float64) + 0.05 * g.standard_normal(workloads.MLP_N_PARAMS))
    theta = theta.astype(np.float32)
    proj = workloads.projections(4, seed=5)
    res = ffc.ffc_compress_tree(cu(Pp), t_g, ffc.Kernel(ffc.GAUSSIAN, h=1.0), tol=1e-6, s0=32, s_max=512,
                                proposal=(cu(theta), cu(proj)))
    out = ffc.tree_result_to_host(res)
    prop = o_compress.Proposal(theta, proj)
    nodes = [i for i in range(t_o.n_nodes) if t_o.level[i] >= 2]
    assert list(out["node"]) == nodes
    swapped = sum(check_learned_node(out, i, Pp, t_o, ko, prop, 1e-6, 32, 512) for i in range(len(nodes)))
    print(f"{len(nodes)} nodes checked, {swapped} rows swapped inside the key margin")


def test_qr_launch_shape_and_autotuner():
    """The QR's launch shape (sub-batch budget, register-resident variant threshold) does not change
    what is computed: across budgets the FP64 ranks, samples, statuses and skeletons are identical
    (integer pivot keys, the same per-column arithmetic) and T and the residual agree to rounding
    (the per-CTA partial sums of ||K'||^2 depend on the column slicing); the tuner returns one of its
    candidates and times every one it tried."""
    from paper_1409_2802_gb300 import autotune
    P = workloads.gaussian_mixture(N=8192, d=8, k=4, seed=11)
    t_g = ffc.ffc_build_tree(cu(P), 256)
    Pp = cu(P)[t_g.perm].contiguous()
    k = ffc.Kernel(ffc.GAUSSIAN, h=1.5)
    outs = [ffc.tree_result_to_host(ffc.ffc_compress_tree(Pp, t_g, k, tol=1e-6, s0=64, s_max=1024,
                                                          qr_l2_budget_mb=b)) for b in (1, 64, 128)]
    for o in outs[1:]:
        for key in ("rank", "s", "status", "skel"):
            assert np.array_equal(outs[0][key], o[key]), key
        assert np.allclose(o["r22_rel"], outs[0]["r22_rel"], rtol=1e-12, atol=1e-300)
        assert np.allclose(o["T"], outs[0]["T"], rtol=1e-9, atol=1e-12 * np.max(np.abs(outs[0]["T"])))
    mixed = [ffc.tree_result_to_host(ffc.ffc_compress_tree(Pp, t_g, k, tol=1e-6, s0=64, s_max=1024,
                                                           precision=ffc.MIXED, qr_big_min_s=b)) for b in (64, 4096)]
    same = mixed[0]["s"] == mixed[1]["s"]          # a tolerance decision at the margin may flip
    assert np.mean(same) >= 0.98
    assert np.max(np.abs(mixed[0]["r22_rel"][same] - mixed[1]["r22_rel"][same])) <= 1e-6
    best = autotune.tune_tree(Pp, t_g, k, precision=ffc.MIXED, tol=1e-6, s0=64, s_max=1024)
    assert best["qr_big_min_s"] in autotune.BIG_MIN_S and best["qr_l2_budget_mb"] in autotune.L2_BUDGET_MB
    assert len(best["table"]) == len(autotune.BIG_MIN_S) + len(autotune.L2_BUDGET_MB) - 1
    assert best["ms"] == min(r.get("ms", float("inf")) for r in best["table"]
                             if r["qr_big_min_s"] == best["qr_big_min_s"])


@pytest.mark.parametrize("precision", [ffc.FP64, ffc.MIXED])
def test_blocked_qr_panels_agree(precision):
    """The QR's panel width changes only rounding: unblocked (1), narrow (2) and wide (8) panels give the
    same samples, ranks, statuses and skeletons in FP64 (integer pivot keys on the same FP64 norms up to
    rounding) and the same residuals and T to rounding; mixed precision agrees within its FP32 rounding."""
    P = workloads.gaussian_mixture(N=8192, d=8, k=4, seed=12)
    t_o = o_tree.build_tree(P, 256)
    t_g = ffc.ffc_build_tree(cu(P), 256)
    Pp = P[t_o.perm]
    k = ffc.Kernel(ffc.GAUSSIAN, h=1.5)
    outs = [ffc.tree_result_to_host(ffc.ffc_compress_tree(cu(Pp), t_g, k, tol=1e-6, s0=64, s_max=1024,
                                                          precision=precision, qr_panel=nb)) for nb in (1, 2, 8)]
    if precision == ffc.FP64:
        for o in outs[1:]:
            for key in ("rank", "s", "status", "skel"):
                assert np.array_equal(outs[0][key], o[key]), key
            # ||R22|| / ||K'|| from FP64 norm downdates in another order: agreement to ~1e-15 of ||K'||
            assert np.max(np.abs(o["r22_rel"] - outs[0]["r22_rel"])) <= 1e-12
            assert np.allclose(o["T"], outs[0]["T"], rtol=1e-7, atol=1e-10 * np.max(np.abs(outs[0]["T"])))
        # and every node against the oracle with the blocked panel
        ko = o_kernels.Kernel(o_kernels.GAUSSIAN, h=1.5)
        nodes = [i for i in range(t_o.n_nodes) if t_o.level[i] >= 2]
        _compare_nodes(outs[2], t_o, Pp, ko, 1e-6, nodes[::2], 64, 1024)
    else:
        for o in outs[1:]:
            same = o["s"] == outs[0]["s"]
            assert np.mean(same) >= 0.98
            assert np.max(np.abs(o["r22_rel"][same] - outs[0]["r22_rel"][same])) <= 1e-6
