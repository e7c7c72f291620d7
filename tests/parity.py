"""Shared parity rules of the GPU tests (imported by the test modules; holds no test).

* ``fp64_error_ok``: the FP64 path's full-block ID error against the oracle's,
  |e_gpu - e_oracle| <= 1e-10 max(e_oracle, 1e-6). Both errors are already
  relative to ||K||_F, so this is 1e-10 relative wherever e >= 1e-6 and
  1e-16 absolute below (the ID's own FP64 rounding).
* ``check_learned_node``: a node compressed with the learned row proposal.
  The draw is checked against the oracle's Efraimidis-Spirakis keys (FP64
  network on FP64 features): every drawn row's key is at or above the s-th
  largest key and every other row's key at or below it, both up to a margin of
  1e-3 of the cut (the FP32 features and logits of the GPU may swap rows whose
  keys are that close, and nothing else). Then the oracle compresses the node
  on the GPU's own ranked rows, and s, status, rank, residual, skeleton and
  full-block error must agree with the GPU's ID as for any other sampler.
"""
from __future__ import annotations

import numpy as np

from oracle import compress as o_compress
from oracle import interp as o_interp
from oracle import mlp as o_mlp
from oracle import proposal as o_prop
from oracle.sampling import far_field_mask

KEY_MARGIN = 1e-3


def fp64_error_tol(e_o: float) -> float:
    return 1e-10 * max(float(e_o), 1e-6)


def fp64_error_ok(e_g: float, e_o: float) -> bool:
    return abs(float(e_g) - float(e_o)) <= fp64_error_tol(e_o)


def node_id(out, i, n):
    """(skel_perm, T (r x (n - r)), r) of output node i of a tree result on the host."""
    r = int(out["rank"][i])
    skel = out["skel"][out["skel_off"][i]: out["skel_off"][i] + n].astype(np.int64)
    T = out["T"][out["T_off"][i]: out["T_off"][i] + r * (n - r)].reshape(n - r, r).T if r else np.zeros((0, n))
    return skel, T, r


def oracle_keys(Pp, t_o, node, kernel_o, proposal: o_compress.Proposal, xi=1.0):
    """(whole-far-field pool, its FP64 keys) of the oracle's learned draw for a node."""
    b, n = int(t_o.begin[node]), int(t_o.count[node])
    far = far_field_mask(Pp, t_o.centroid[node], t_o.radius[node], xi, b, b + n)
    pool = np.flatnonzero(far)
    F = o_prop.features(Pp, pool, t_o.centroid[node], t_o.radius[node], kernel_o, proposal.proj)
    o, _ = o_mlp.forward(o_mlp.half_weights(proposal.theta32), F)
    return pool, o_prop.es_keys(o_prop.mixed_weights(o), 0, node)


def check_draw(rows, pool, keys, s):
    """The s drawn rows are the s best keys of the pool up to KEY_MARGIN of the cut."""
    rows = np.asarray(rows, dtype=np.int64)
    assert rows.size == min(s, pool.size) and np.unique(rows).size == rows.size
    pos = np.searchsorted(pool, rows)
    assert np.all(pos < pool.size) and np.array_equal(pool[pos], rows), "a drawn row is not in the far field"
    if rows.size == pool.size:
        return 0
    cut = np.sort(keys)[::-1][rows.size - 1]
    margin = KEY_MARGIN * abs(cut)
    assert np.min(keys[pos]) >= cut - margin, "a drawn row's key is below the cut"
    rest = np.ones(pool.size, dtype=bool)
    rest[pos] = False
    assert np.max(keys[rest]) <= cut + margin, "an undrawn row's key is above the cut"
    best = np.argsort(-keys, kind="stable")[:rows.size]
    return int(rows.size - np.intersect1d(pool[best], rows).size)   # rows swapped inside the margin


def far_rows_subset(Pp64, t_o, node, k_near=2048, k_uniform=2048, seed=0):
    """Far-field rows nearest to the node centroid (they carry a Laplace block) plus a seeded
    uniform pick of the rest: the rows on which both IDs' full-block errors are compared when the
    whole far field is too large for the oracle."""
    b, n = int(t_o.begin[node]), int(t_o.count[node])
    far = np.flatnonzero(far_field_mask(Pp64, t_o.centroid[node], t_o.radius[node], 1.0, b, b + n))
    dist = np.sum((Pp64[far] - t_o.centroid[node]) ** 2, axis=1)
    order = np.argsort(dist, kind="stable")
    near = far[order[:k_near]]
    rest = far[order[k_near:]]
    pick = np.random.default_rng(seed + node).choice(rest, min(k_uniform, rest.size), replace=False) \
        if rest.size else rest
    return np.sort(np.concatenate([near, pick]))


def check_learned_node(out, i, Pp, t_o, kernel_o, proposal, tol, s0, s_max, err_rows=None, precision_fp64=True):
    """Draw and ID of output node i (see the module docstring). Returns the number of swapped rows."""
    node = int(out["node"][i])
    b, n = int(t_o.begin[node]), int(t_o.count[node])
    s = int(out["s"][i])
    pool, keys = oracle_keys(Pp, t_o, node, kernel_o, proposal)
    ranked = out["rows"][out["rows_off"][i]: out["rows_off"][i] + min(s_max, pool.size)]
    swapped = check_draw(ranked[:s], pool, keys, s)
    ref = o_compress.compress_node(Pp, t_o, node, kernel_o, tol, 0, s0, s_max, ranked_rows=ranked)
    assert s == ref.s, (node, s, ref.s)
    skel, T, r = node_id(out, i, n)
    P_g = o_interp.assemble_P(skel, T, n)
    assert np.array_equal(P_g[:, skel[:r]], np.eye(r))
    if precision_fp64:
        assert int(out["status"][i]) == ref.status and r == ref.rank, (node, r, ref.rank)
        assert abs(out["r22_rel"][i] - ref.r22_rel) <= 1e-10, node
        sub = err_rows if err_rows is not None else far_field_mask(Pp, t_o.centroid[node], t_o.radius[node], 1.0,
                                                                   b, b + n)
        e_g = o_interp.full_block_error(kernel_o, Pp[sub], Pp[b:b + n], skel, T)
        e_o = o_interp.full_block_error(kernel_o, Pp[sub], Pp[b:b + n], ref.skel_perm, ref.T)
        assert fp64_error_ok(e_g, e_o), (node, e_g, e_o)
    return swapped
