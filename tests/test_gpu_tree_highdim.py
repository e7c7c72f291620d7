"""GPU parity of the tree path on the d = 128 and d = 1,000 workloads, at full size.

* d = 128: N = 262,144 points of the decaying 16-component mixture (seed 1000),
  leaf 256 (levels 2..10, 2,044 nodes); Laplace |x - y|^-126 and the cubic
  polynomial (x.y / 128 + 1)^3.
* d = 1,000: N = 100,000 points of intrinsic dimension 10 plus N(0, 0.01^2)
  noise (seed 1000), stored in FP32; leaf 512 (levels 2..8, 508 nodes);
  Gaussian with h = the median pairwise distance of a 4,096-point subset.

Both precisions run over the whole tree (s = 128 doubling to 2,048, tol 1e-6),
in the launch configuration the benchmark times. Every node is checked for the
properties that hold at any size; a seeded sample of nodes of the deepest
levels (the ones the oracle finishes in seconds) is compressed by the oracle.
The full-block error of an ID is evaluated by the oracle on a fixed subset of
the far field (its rows nearest to the centroid, which carry the Laplace
block, plus a seeded uniform pick), the same rows for the GPU's and the
oracle's ID.
"""
import numpy as np
import pytest
import torch

import workloads
from oracle import compress as o_compress
from oracle import interp as o_interp
from oracle import kernels as o_kernels
from oracle import tree as o_tree
from oracle.sampling import far_field_mask
from parity import check_learned_node, far_rows_subset, fp64_error_ok, node_id

pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_1409_2802_gb300 import ffc  # noqa: E402

DEV = torch.device("cuda:0")
TOL, S0, S_MAX = 1e-6, 128, 2048


def cu(a):
    return torch.tensor(np.ascontiguousarray(a), device=DEV)


class Workload:
    def __init__(self, P, leaf):
        self.P = P
        self.t_o = o_tree.build_tree(P, leaf)
        self.t_g = ffc.ffc_build_tree(cu(P), leaf)
        self.Pp = P[self.t_o.perm]                   # stored precision (FP64 or FP32)
        self.Pp64 = self.Pp.astype(np.float64)
        self.Pp_dev = cu(self.Pp)


@pytest.fixture(scope="module")
def d128():
    return Workload(workloads.decaying_mixture(N=262144, d=128, k=16, seed=1000), 256)


@pytest.fixture(scope="module")
def d1000():
    return Workload(workloads.low_intrinsic(N=100000, d_i=10, d_e=1000, seed=1000), 512)


def _check_tree(w):
    t_o, t_g = w.t_o, w.t_g
    assert t_g.depth == t_o.depth
    assert np.array_equal(t_g.perm.cpu().numpy(), t_o.perm)
    assert np.array_equal(t_g.begin.cpu().numpy(), t_o.begin)
    assert np.array_equal(t_g.count.cpu().numpy(), t_o.count)
    scale = max(1.0, float(np.abs(t_o.centroid).max()))
    np.testing.assert_allclose(t_g.centroid.cpu().numpy(), t_o.centroid, rtol=0, atol=1e-12 * scale)
    np.testing.assert_allclose(t_g.radius.cpu().numpy(), t_o.radius, rtol=1e-12)


def test_tree_d128_matches_oracle(d128):
    _check_tree(d128)


def test_tree_d1000_fp32_matches_oracle(d1000):
    _check_tree(d1000)


def _invariants(out, t_o):
    nodes = [i for i in range(t_o.n_nodes) if t_o.level[i] >= 2]
    assert list(out["node"]) == nodes
    st = out["status"]
    assert np.all((st == 0) | (st == ffc.FFC_E_TOL_NOT_REACHED))
    assert np.all(out["r22_rel"][st == 0] <= TOL)
    n = t_o.count[out["node"]]
    assert np.all(out["rank"] <= np.minimum(n, S_MAX // 2))
    for i in range(len(nodes)):
        skel = out["skel"][out["skel_off"][i]: out["skel_off"][i] + n[i]]
        assert np.array_equal(np.sort(skel), np.arange(n[i])), nodes[i]


def _rows_subset(Pp64, t_o, node):
    return far_rows_subset(Pp64, t_o, node)


def _id_of(out, i, n):
    return node_id(out, i, n)


def _compare(w, out, ko, nodes, precision):
    index = {int(nd): i for i, nd in enumerate(out["node"])}
    for node in nodes:
        i = index[node]
        ref = o_compress.compress_node(w.Pp64, w.t_o, node, ko, TOL, 0, S0, S_MAX)
        s = int(out["s"][i])
        n, b = int(w.t_o.count[node]), int(w.t_o.begin[node])
        skel, T, r = _id_of(out, i, n)
        P_g = o_interp.assemble_P(skel, T, n)
        assert np.array_equal(P_g[:, skel[:r]], np.eye(r))
        if precision == ffc.FP64 or s == ref.s:
            assert s == ref.s, node
            rows = out["rows"][out["rows_off"][i]: out["rows_off"][i] + s]
            assert np.array_equal(rows, ref.rows), node
        sub = _rows_subset(w.Pp64, w.t_o, node)
        e_g = o_interp.full_block_error(ko, w.Pp64[sub], w.Pp64[b:b + n], skel, T)
        e_o = o_interp.full_block_error(ko, w.Pp64[sub], w.Pp64[b:b + n], ref.skel_perm, ref.T)
        if precision == ffc.FP64:
            assert int(out["status"][i]) == ref.status, node
            assert r == ref.rank, (node, r, ref.rank)
            assert abs(out["r22_rel"][i] - ref.r22_rel) <= 1e-10, node
            assert fp64_error_ok(e_g, e_o), (node, e_g, e_o, abs(e_g - e_o))
        else:
            assert abs(e_g - e_o) <= max(1e-6, 1e-4 * e_o), (node, e_g, e_o)


def _deep_nodes(t_o, count, levels, seed):
    cand = [i for i in range(t_o.n_nodes) if t_o.level[i] in levels]
    return sorted(np.random.default_rng(seed).choice(cand, count, replace=False).tolist())


@pytest.mark.parametrize("precision", [ffc.FP64, ffc.MIXED])
@pytest.mark.parametrize("kind", ["laplace", "polynomial"])
def test_compress_d128_full_size(d128, kind, precision):
    w = d128
    if kind == "laplace":
        kg, ko = ffc.Kernel(ffc.LAPLACE), o_kernels.Kernel(o_kernels.LAPLACE)
        levels = (8, 9, 10)
    else:
        kg = ffc.Kernel(ffc.POLYNOMIAL, h=128.0, c=1.0, p=3)
        ko = o_kernels.Kernel(o_kernels.POLYNOMIAL, h=128.0, c=1.0, p=3)
        levels = (9, 10)
    out = ffc.tree_result_to_host(ffc.ffc_compress_tree(w.Pp_dev, w.t_g, kg, tol=TOL, precision=precision, s0=S0,
                                                        s_max=S_MAX))
    assert out["n_out"] == 2044
    _invariants(out, w.t_o)
    _compare(w, out, ko, _deep_nodes(w.t_o, 3, levels, seed=11 + precision), precision)


@pytest.mark.parametrize("precision", [ffc.FP64, ffc.MIXED])
def test_compress_d1000_fp32_full_size(d1000, precision):
    w = d1000
    h = workloads.median_pairwise_distance(w.P)
    kg, ko = ffc.Kernel(ffc.GAUSSIAN, h=h), o_kernels.Kernel(o_kernels.GAUSSIAN, h=h)
    out = ffc.tree_result_to_host(ffc.ffc_compress_tree(w.Pp_dev, w.t_g, kg, tol=TOL, precision=precision, s0=S0,
                                                        s_max=S_MAX))
    assert out["n_out"] == 508
    _invariants(out, w.t_o)
    _compare(w, out, ko, _deep_nodes(w.t_o, 2, (8,), seed=21 + precision), precision)


@pytest.mark.parametrize("which", ["d128_laplace", "d1000"])
def test_compress_learned_sampler_full_size(d128, d1000, which):
    """Learned sampler with a seeded (untrained) network: every node's rows are
    distinct far-field rows; on sampled leaves the draw is the oracle's best keys up
    to the FP32 logits' rounding, and the ID on the drawn rows is the oracle's."""
    if which == "d128_laplace":
        w, kg, ko = d128, ffc.Kernel(ffc.LAPLACE), o_kernels.Kernel(o_kernels.LAPLACE)
    else:
        w = d1000
        h = workloads.median_pairwise_distance(w.P)
        kg, ko = ffc.Kernel(ffc.GAUSSIAN, h=h), o_kernels.Kernel(o_kernels.GAUSSIAN, h=h)
    d = w.P.shape[1]
    g = np.random.default_rng(3)
    theta = (workloads.mlp_init(9).astype(np.float64) + 0.05 * g.standard_normal(workloads.MLP_N_PARAMS))
    theta = theta.astype(np.float32)
    proj = workloads.projections(d, seed=5)
    out = ffc.tree_result_to_host(ffc.ffc_compress_tree(w.Pp_dev, w.t_g, kg, tol=TOL, precision=ffc.FP64, s0=S0,
                                                        s_max=S_MAX, proposal=(cu(theta), cu(proj))))
    _invariants(out, w.t_o)
    index = {int(nd): i for i, nd in enumerate(out["node"])}
    g2 = np.random.default_rng(4)
    for i in sorted(g2.choice(len(out["node"]), 16, replace=False).tolist()):
        node = int(out["node"][i])
        b, n = int(w.t_o.begin[node]), int(w.t_o.count[node])
        s = int(out["s"][i])
        rows = out["rows"][out["rows_off"][i]: out["rows_off"][i] + s]
        far = far_field_mask(w.Pp64, w.t_o.centroid[node], w.t_o.radius[node], 1.0, b, b + n)
        assert np.unique(rows).size == s and np.all(far[rows]), node
    prop = o_compress.Proposal(theta, proj)
    swapped = 0
    for node in _deep_nodes(w.t_o, 4, (w.t_o.depth,), seed=31):
        i = index[node]
        swapped += check_learned_node(out, i, w.Pp64, w.t_o, ko, prop, TOL, S0, S_MAX,
                                      err_rows=_rows_subset(w.Pp64, w.t_o, node))
    print(f"4 leaves checked, {swapped} rows swapped inside the key margin")

