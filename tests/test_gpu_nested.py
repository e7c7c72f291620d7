"""GPU parity of nested skeletonization (ffc_params.nested): the upward pass whose node IDs take their
children's skeleton points as columns, against the oracle (oracle/compress.compress_tree_nested), and
the evaluation from the nested representations (ffc_tree_apply) against oracle/apply.

FP64: a node's columns are built from its children's skeletons, which the plain parity tests show equal
to the oracle's, so columns, samples, ranks, skeletons and statuses are compared exactly; the ID's error
on its full far-field block (against the columns) to 1e-10 max(e, 1e-6); potentials to 1e-9 of the
largest (the two sides' T agree to rounding).
"""
import numpy as np
import pytest
import torch

import workloads
from oracle import apply as o_apply
from oracle import compress as o_compress
from oracle import interp as o_interp
from oracle import kernels as o_kernels
from oracle import tree as o_tree
from oracle.sampling import far_field_mask
from parity import fp64_error_ok, node_id

pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_1409_2802_gb300 import ffc  # noqa: E402

DEV = torch.device("cuda:0")
S0, S_MAX = 32, 512


def cu(a):
    return torch.tensor(np.ascontiguousarray(a), device=DEV)


def _case(N=4096, d=4, leaf=256, seed=2):
    P = workloads.gaussian_mixture(N=N, d=d, k=4, seed=seed)
    t_o = o_tree.build_tree(P, leaf)
    t_g = ffc.ffc_build_tree(cu(P), leaf)
    return P[t_o.perm], t_o, t_g


def _kernels(which):
    if which == "gaussian":
        return o_kernels.Kernel(o_kernels.GAUSSIAN, h=1.0), ffc.Kernel(ffc.GAUSSIAN, h=1.0)
    if which == "laplace":
        return o_kernels.Kernel(o_kernels.LAPLACE), ffc.Kernel(ffc.LAPLACE)
    return (o_kernels.Kernel(o_kernels.POLYNOMIAL, h=4.0, c=1.0, p=3),
            ffc.Kernel(ffc.POLYNOMIAL, h=4.0, c=1.0, p=3))


@pytest.mark.parametrize("which", ["gaussian", "laplace"])
def test_nested_compression_matches_oracle(which):
    Pp, t_o, t_g = _case()
    ko, kg = _kernels(which)
    res = ffc.ffc_compress_tree(cu(Pp), t_g, kg, tol=1e-6, s0=S0, s_max=S_MAX, nested=True)
    out = ffc.tree_result_to_host(res)
    ref = o_compress.compress_tree_nested(Pp, t_o, ko, 1e-6, s0=S0, s_max=S_MAX)
    for i, node in enumerate(out["node"]):
        node = int(node)
        rf = ref[node]
        nc = int(out["ncols"][i])
        cols = out["cols"][out["skel_off"][i]: out["skel_off"][i] + nc]
        assert np.array_equal(cols, rf.cols), node
        s = int(out["s"][i])
        assert s == rf.s and int(out["status"][i]) == rf.status, node
        rows = out["rows"][out["rows_off"][i]: out["rows_off"][i] + s]
        assert np.array_equal(rows, rf.rows), node
        skel, T, r = node_id(out, i, nc)
        assert r == rf.rank and np.array_equal(skel[:r], rf.skel_perm[:r]), node
        assert abs(out["r22_rel"][i] - rf.r22_rel) <= 1e-10, node
        if r == 0:
            continue
        b, n = int(t_o.begin[node]), int(t_o.count[node])
        far = far_field_mask(Pp, t_o.centroid[node], t_o.radius[node], 1.0, b, b + n)
        Xc = Pp[b + cols]
        e_g = o_interp.full_block_error(ko, Pp[far], Xc, skel, T)
        e_o = o_interp.full_block_error(ko, Pp[far], Xc, rf.skel_perm, rf.T)
        assert fp64_error_ok(e_g, e_o), (node, e_g, e_o)
    # internal nodes have fewer columns than points (their children compress)
    lv = np.floor(np.log2(out["node"] + 1)).astype(int)
    inner = lv < t_o.depth
    assert np.all(out["ncols"][inner] <= t_o.count[out["node"][inner]])
    assert np.any(out["ncols"][inner] < t_o.count[out["node"][inner]])


@pytest.mark.parametrize("which", ["gaussian", "polynomial"])
def test_nested_tree_apply_matches_oracle(which):
    Pp, t_o, t_g = _case(seed=3)
    ko, kg = _kernels(which)
    res = ffc.ffc_compress_tree(cu(Pp), t_g, kg, tol=1e-10 if which == "polynomial" else 1e-6, s0=S0,
                                s_max=S_MAX, nested=True)
    ref = o_compress.compress_tree_nested(Pp, t_o, ko, 1e-10 if which == "polynomial" else 1e-6, s0=S0,
                                          s_max=S_MAX)
    q = np.random.default_rng(4).standard_normal(len(Pp))
    u_g, _ = ffc.ffc_tree_apply(cu(Pp), t_g, res, cu(q), mode=ffc.APPLY_SKELETON, s_max=S_MAX)
    u_g = u_g.cpu().numpy()
    u_o = o_apply.nested_tree_potential(ko, Pp, t_o, q, ref)
    assert np.max(np.abs(u_g - u_o)) <= 1e-9 * np.max(np.abs(u_o))
    if which == "polynomial":
        # a cubic in d = 4 has exact rank C(7, 3) = 35: nested representations are exact at every level
        u_d = o_apply.tree_potential(ko, Pp, t_o, q, mode="direct")
        assert np.max(np.abs(u_g - u_d)) <= 1e-8 * np.max(np.abs(u_d))


def test_plain_call_after_nested_resets_the_columns():
    Pp, t_o, t_g = _case(seed=5)
    ko, kg = _kernels("gaussian")
    fresh = ffc.tree_result_to_host(ffc.ffc_compress_tree(cu(Pp), t_g, kg, tol=1e-6, s0=S0, s_max=S_MAX))
    res = ffc.ffc_compress_tree(cu(Pp), t_g, kg, tol=1e-6, s0=S0, s_max=S_MAX, nested=True)
    again = ffc.tree_result_to_host(ffc.ffc_compress_tree(cu(Pp), t_g, kg, tol=1e-6, s0=S0, s_max=S_MAX, result=res))
    for key in ("rank", "s", "status", "skel", "T", "ncols", "cols"):
        assert np.array_equal(fresh[key], again[key]), key
    assert np.array_equal(again["ncols"], t_o.count[again["node"]])


def test_nested_mixed_precision_runs_the_full_size_d16_tree():
    """The benchmark tree (N = 65,536, d = 16, Gaussian h = 2) in mixed precision, nested: every node's
    columns are its children's skeleton points, and statuses and residuals obey the tolerance."""
    P = workloads.gaussian_mixture(N=65536, d=16, k=8, seed=0)
    t_g = ffc.ffc_build_tree(cu(P), 256)
    Pp = cu(P)[t_g.perm].contiguous()
    out = ffc.tree_result_to_host(ffc.ffc_compress_tree(Pp, t_g, ffc.Kernel(ffc.GAUSSIAN, h=2.0), tol=1e-6,
                                                        precision=ffc.MIXED, s0=128, s_max=2048, nested=True))
    st = out["status"]
    assert np.all((st == 0) | (st == ffc.FFC_E_TOL_NOT_REACHED))
    assert np.all(out["r22_rel"][st == 0] <= 1e-6)
    count = t_g.count.cpu().numpy()
    first = int(out["node"][0])
    for i, node in enumerate(out["node"]):
        node = int(node)
        if 2 * node + 2 >= len(count):
            continue
        want = 0
        for ch in (2 * node + 1, 2 * node + 2):
            oc = ch - first
            want += int(out["rank"][oc]) if (int(out["status"][oc]) in (0, 7) and int(out["s"][oc]) > 0) \
                else int(count[ch])
        assert int(out["ncols"][i]) == want, node
