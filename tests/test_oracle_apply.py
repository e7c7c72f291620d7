"""Pins of the outgoing-representation oracle (§2.1.3: q~ = P q, u ~ C q~).

* A full-rank ID (r = n) represents the block exactly, so C q~ is K q.
* For any ID, |K q - C P q| <= ||K - C P||_2 ||q|| <= ||K - C P||_F ||q||.
* Low-rank blocks: with a polynomial kernel of exact rank C(d + p, p), the
  representation at that rank reproduces K q to rounding.
"""
import math

import numpy as np

import workloads
from oracle import apply as o_apply
from oracle import interp as o_interp
from oracle import kernels as o_kernels


def _id(K, r_max, tol=0.0):
    ref = o_interp.interpolative_decomposition(K, r_max, tol)
    return ref["skel_perm"], ref["T"], ref["rank"]


def test_full_rank_representation_is_exact():
    X, Y = workloads.single_block(0, n=64, m=200)
    k = o_kernels.Kernel(o_kernels.GAUSSIAN, h=1.0)
    K, _ = o_kernels.kernel_block(k, Y, X)
    skel, T, r = _id(K, 64)
    assert r == 64 and T.shape == (64, 0)
    q = np.random.default_rng(1).standard_normal(64)
    qt = o_apply.skeleton_charges(skel, T, q)
    assert np.array_equal(qt, q[skel[:64]])
    u, _ = o_apply.direct_potential(k, Y, X, q)
    ut, _ = o_apply.id_potential(k, Y, X, skel, r, qt)
    assert np.max(np.abs(u - ut)) <= 1e-12 * np.max(np.abs(u))


def test_error_within_the_block_error_times_the_charges():
    X, Y = workloads.single_block(0)
    k = o_kernels.Kernel(o_kernels.GAUSSIAN, h=1.0)
    K, _ = o_kernels.kernel_block(k, Y, X)
    g = np.random.default_rng(2)
    for r_max in (8, 32, 64):
        skel, T, r = _id(K, r_max)
        P = o_interp.assemble_P(skel, T, K.shape[1])
        E = K - K[:, skel[:r]] @ P
        for _ in range(3):
            q = g.standard_normal(K.shape[1])
            qt = o_apply.skeleton_charges(skel, T, q)
            u, _ = o_apply.direct_potential(k, Y, X, q)
            ut, _ = o_apply.id_potential(k, Y, X, skel, r, qt)
            err = np.linalg.norm(u - ut)
            assert err <= np.linalg.norm(E, 2) * np.linalg.norm(q) * (1 + 1e-9) + 1e-12
            assert err <= np.linalg.norm(E) * np.linalg.norm(q) * (1 + 1e-9) + 1e-12


def test_polynomial_exact_rank_reproduces_the_potential():
    d, p = 3, 2
    g = np.random.default_rng(3)
    X = g.standard_normal((40, d))
    Y = g.standard_normal((90, d))
    k = o_kernels.Kernel(o_kernels.POLYNOMIAL, h=2.0, c=1.0, p=p)
    K, _ = o_kernels.kernel_block(k, Y, X)
    rank = math.comb(d + p, p)
    skel, T, r = _id(K, rank)
    q = g.standard_normal(40)
    u, _ = o_apply.direct_potential(k, Y, X, q)
    ut, _ = o_apply.id_potential(k, Y, X, skel, r, o_apply.skeleton_charges(skel, T, q))
    assert r == rank
    assert np.max(np.abs(u - ut)) <= 1e-9 * np.max(np.abs(u))


def test_laplace_potentials_share_the_scale():
    X, Y = workloads.single_block(1, n=48, m=120, d=5)
    Y = Y + 2.0
    k = o_kernels.Kernel(o_kernels.LAPLACE)
    K, _ = o_kernels.kernel_block(k, Y, X)
    skel, T, r = _id(K, 48)
    q = np.random.default_rng(4).standard_normal(48)
    u, lu = o_apply.direct_potential(k, Y, X, q)
    ut, lt = o_apply.id_potential(k, Y, X, skel, r, o_apply.skeleton_charges(skel, T, q))
    assert lu == lt
    assert np.max(np.abs(u - ut)) <= 1e-10 * np.max(np.abs(u))
