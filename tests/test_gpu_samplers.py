"""GPU parity of the paper's other row samplers (§4.1.3; §3 heuristics) against the oracle:
distance sampling in both readings, nearest neighbours and leverage sampling.

Both sides compute FP64 distances (in different summation orders) and draw the
same Philox stream, so the draws agree except where two keys (or two nearest
distances) tie to rounding: every drawn row's oracle key is at or above the
s-th best key and every other row's at or below it, within a margin of 1e-12
of the cut (distance samplers, nearest neighbours). Leverage scores carry the
eigen-solver's error (a Davis-Kahan bound of about 1e-10 on these blocks), so
their keys get a margin of 1e-6.
"""
import numpy as np
import pytest
import torch

import workloads
from oracle import kernels as o_kernels
from oracle import samplers as o_samp
from oracle import spectral as o_spec
from oracle.sampling import far_field_mask

pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_1409_2802_gb300 import ffc  # noqa: E402

DEV = torch.device("cuda:0")


def cu(a):
    return torch.tensor(np.ascontiguousarray(a), device=DEV)


def _node(N, d, n, seed):
    """Points sorted by distance to the first one; the node is the first n, its far field the candidates."""
    Y = workloads.gaussian_mixture(N, d, 4, seed=seed)
    Y = Y[np.argsort(np.sum((Y - Y[0]) ** 2, axis=1), kind="stable")]
    x_c = Y[:n].mean(axis=0)
    rho = float(np.sqrt(np.max(np.sum((Y[:n] - x_c) ** 2, axis=1))))
    cand = np.flatnonzero(far_field_mask(Y, x_c, rho, 1.0, 0, n))
    return np.ascontiguousarray(Y), x_c, cand


def _check_ranked(rows, cand, score, s, margin_rel, larger_first=True):
    """rows = the best min(s, P) candidates by score up to margin_rel of the cut; returns swaps."""
    rows = np.asarray(rows)
    keep = min(s, cand.size)
    assert rows.size == keep and np.unique(rows).size == keep
    pos = np.searchsorted(cand, rows)
    assert np.all(pos < cand.size) and np.array_equal(cand[pos], rows)
    sc = score if larger_first else -score
    if keep == cand.size:
        return 0
    cut = np.sort(sc)[::-1][keep - 1]
    margin = margin_rel * abs(cut)
    assert np.min(sc[pos]) >= cut - margin
    rest = np.ones(cand.size, bool)
    rest[pos] = False
    assert np.max(sc[rest]) <= cut + margin
    best = np.argsort(-sc, kind="stable")[:keep]
    return int(keep - np.intersect1d(cand[best], rows).size)


@pytest.mark.parametrize("sampler", [ffc.DRAW_DISTANCE, ffc.DRAW_INV_DISTANCE])
@pytest.mark.parametrize("N,s", [(4096, 300), (40000, 2048), (2000, 5000), (30000, 7)])
def test_distance_samplers_match_oracle(sampler, N, s):
    Y, x_c, cand = _node(N, 8, 128, seed=N + s)
    inverse = sampler == ffc.DRAW_INV_DISTANCE
    rows_o, keys = o_samp.weighted_draw(cand, o_samp.distance_weights(Y, cand, x_c, inverse), s, 3, 17)
    rows_g = ffc.ffc_sample_paper(sampler, cu(Y), cu(cand), s, 3, 17, x_c=cu(x_c)).cpu().numpy()
    if not np.array_equal(rows_g, rows_o):
        _check_ranked(rows_g, cand, keys, s, 1e-12)
    # a size-s draw is a prefix of the size-2s draw
    rows_2 = ffc.ffc_sample_paper(sampler, cu(Y), cu(cand), 2 * s, 3, 17, x_c=cu(x_c)).cpu().numpy()
    assert list(rows_2[:rows_g.size]) == list(rows_g)


@pytest.mark.parametrize("N,n,s", [(4096, 128, 200), (20000, 700, 1000), (1000, 64, 2000)])
def test_nearest_neighbours_match_oracle(N, n, s):
    Y, x_c, cand = _node(N, 6, n, seed=n)
    rows_o = o_samp.nearest_neighbours(Y, cand, Y[:n], s)
    rows_g = ffc.ffc_sample_paper(ffc.DRAW_NEAREST, cu(Y), cu(cand), s, 0, 0, X=cu(Y[:n])).cpu().numpy()
    if not np.array_equal(rows_g, rows_o):
        dmin = np.min(np.sum((Y[cand][:, None, :] - Y[None, :n, :]) ** 2, axis=2), axis=1)
        _check_ranked(rows_g, cand, dmin, s, 1e-12, larger_first=False)


@pytest.mark.parametrize("kind", [o_kernels.GAUSSIAN, o_kernels.LAPLACE])
def test_leverage_sampling_matches_oracle(kind):
    Y, x_c, cand = _node(6000, 5, 200, seed=11)
    k = o_kernels.Kernel(kind, h=1.0)
    K, _ = o_kernels.kernel_block(k, Y[cand], Y[:200])
    eps = 1e-6
    r_o = o_spec.eps_rank(K, eps)
    for s in (64, 256):
        rows_o = o_samp.leverage_sample(K, cand, s, eps, 5, 9)
        rows_g, r_g, st = ffc.ffc_sample_leverage(cu(K.T.copy()), s, 5, 9, eps=eps, cand=cu(cand))
        rows_g = rows_g.cpu().numpy()
        assert r_g == r_o and st == ffc.FFC_OK
        if not np.array_equal(rows_g, rows_o):
            lev = o_spec.row_leverage_scores(K, r_o)
            keep = lev > 0
            _, keys = o_samp.weighted_draw(cand[keep], lev[keep], s, 5, 9)
            _check_ranked(rows_g, cand[keep], keys, s, 1e-6)


def test_samplers_reject_bad_arguments():
    Y = cu(np.zeros((10, 3)))
    cand = cu(np.arange(10))
    with pytest.raises(ffc.FFCError):
        ffc.ffc_sample_paper(7, Y, cand, 3, 0, 0, x_c=cu(np.zeros(3)))
    with pytest.raises(ffc.FFCError):
        ffc.ffc_sample_paper(ffc.DRAW_NEAREST, Y, cand, 3, 0, 0)           # no sources


@pytest.mark.parametrize("which", ["distance", "inv_distance", "nearest"])
def test_tree_paper_samplers_match_oracle(which):
    """ffc_compress_tree with a paper sampler, FP64, every node: the drawn rows are the oracle's draw
    over the node's far field (up to ties within 1e-12), and the ID on the drawn rows is the oracle's."""
    from oracle import compress as o_compress
    from oracle import interp as o_interp
    from oracle import tree as o_tree
    from parity import fp64_error_ok, node_id
    P = workloads.gaussian_mixture(N=4096, d=4, k=4, seed=8)
    t_o = o_tree.build_tree(P, 256)
    t_g = ffc.ffc_build_tree(cu(P), 256)
    Pp = P[t_o.perm]
    ko = o_kernels.Kernel(o_kernels.GAUSSIAN, h=1.0)
    code = {"distance": ffc.SAMPLE_DISTANCE, "inv_distance": ffc.SAMPLE_INV_DISTANCE,
            "nearest": ffc.SAMPLE_NEAREST}[which]
    s0, s_max = 32, 512
    out = ffc.tree_result_to_host(ffc.ffc_compress_tree(cu(Pp), t_g, ffc.Kernel(ffc.GAUSSIAN, h=1.0), tol=1e-6,
                                                        s0=s0, s_max=s_max, sampler=code))
    for i, node in enumerate(out["node"]):
        node = int(node)
        b, n = int(t_o.begin[node]), int(t_o.count[node])
        far = far_field_mask(Pp, t_o.centroid[node], t_o.radius[node], 1.0, b, b + n)
        cand = np.flatnonzero(far)
        s = int(out["s"][i])
        ranked = out["rows"][out["rows_off"][i]: out["rows_off"][i] + min(s_max, cand.size)]
        if which == "nearest":
            dmin = np.min(np.sum((Pp[cand][:, None, :] - Pp[None, b:b + n, :]) ** 2, axis=2), axis=1)
            _check_ranked(ranked[:s], cand, dmin, s, 1e-12, larger_first=False)
        else:
            w = o_samp.distance_weights(Pp, cand, t_o.centroid[node], inverse=which == "inv_distance")
            _, keys = o_samp.weighted_draw(cand, w, s, 0, node)
            _check_ranked(ranked[:s], cand, keys, s, 1e-12)
        ref = o_compress.compress_node(Pp, t_o, node, ko, 1e-6, 0, s0, s_max, ranked_rows=ranked)
        assert s == ref.s and int(out["status"][i]) == ref.status and int(out["rank"][i]) == ref.rank, node
        skel, T, r = node_id(out, i, n)
        e_g = o_interp.full_block_error(ko, Pp[far], Pp[b:b + n], skel, T)
        e_o = o_interp.full_block_error(ko, Pp[far], Pp[b:b + n], ref.skel_perm, ref.T)
        assert fp64_error_ok(e_g, e_o), (node, e_g, e_o)
