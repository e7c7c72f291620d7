"""Pins of the learned-proposal oracle (network, loss, Adam, weighted sampling,
features, leverage targets) against closed forms, finite differences and
exact probabilities."""
import math

import numpy as np
import pytest

import workloads
from oracle import mlp, proposal
from oracle.kernels import GAUSSIAN, LAPLACE, POLYNOMIAL, Kernel
from oracle.sampling import far_field_mask, sample_uniform_from_mask
from oracle.spectral import eps_rank


def test_layout_matches_generator():
    assert mlp.N_PARAMS == workloads.MLP_N_PARAMS
    assert mlp.LAYOUT == workloads.MLP_LAYOUT
    offs = sorted(mlp.LAYOUT.values())
    end = 0
    for off, shape in offs:
        assert off == end
        end = off + int(np.prod(shape))
    assert end == mlp.N_PARAMS


def test_gelu_closed_forms():
    # Phi(1) = 0.8413447460685429 (standard normal table)
    assert mlp.gelu(np.array(0.0)) == 0.0
    assert abs(mlp.gelu(np.array(1.0)) - 0.8413447460685429) < 1e-15
    assert abs(mlp.gelu(np.array(-1.0)) + 0.15865525393145707) < 1e-15
    z = np.linspace(-6, 6, 101)
    # z Phi(z) - (-z) Phi(-z) = z (Phi(z) + Phi(-z)) = z
    assert np.max(np.abs(mlp.gelu(z) - mlp.gelu(-z) - z)) < 1e-14
    assert abs(mlp.gelu_prime(np.array(0.0)) - 0.5) < 1e-15
    h = 1e-5
    fd = (mlp.gelu(z + h) - mlp.gelu(z - h)) / (2 * h)
    assert np.max(np.abs(fd - mlp.gelu_prime(z))) < 1e-9


def _small_problem(seed=3, R=37):
    g = np.random.default_rng(seed)
    theta = g.standard_normal(mlp.N_PARAMS) * 0.3
    X = g.standard_normal((R, 12))
    off = np.array([0, 15, R])
    t = g.random(R)
    for b in range(2):
        t[off[b]:off[b + 1]] /= t[off[b]:off[b + 1]].sum()
    return theta, X, t, off


def test_backward_matches_central_differences():
    theta, X, t, off = _small_problem()
    loss, grad = mlp.loss_and_grad(theta, X, t, off, half=False)
    g = np.random.default_rng(7)
    coords = [mlp.LAYOUT["b3"][0]]
    for name, (o, shape) in mlp.LAYOUT.items():
        size = int(np.prod(shape))
        coords += list(o + g.choice(size, size=min(size, 12), replace=False))
    h = 1e-6
    for c in coords:
        tp = theta.copy(); tp[c] += h
        tm = theta.copy(); tm[c] -= h
        lp, _ = mlp.loss_and_grad(tp, X, t, off, half=False)
        lm, _ = mlp.loss_and_grad(tm, X, t, off, half=False)
        fd = (lp - lm) / (2 * h)
        assert abs(fd - grad[c]) <= 1e-7 + 1e-6 * abs(grad[c]), (c, fd, grad[c])


def test_cross_entropy_properties():
    g = np.random.default_rng(11)
    o = g.standard_normal(20)
    off = np.array([0, 8, 20])
    # targets equal to the per-node softmax: zero gradient, loss = mean entropy
    t = np.empty(20)
    ent = 0.0
    for b in range(2):
        ob = o[off[b]:off[b + 1]]
        p = np.exp(ob - ob.max()); p /= p.sum()
        t[off[b]:off[b + 1]] = p
        ent += -np.sum(p * np.log(p))
    loss, g_o = mlp.softmax_cross_entropy(o, t, off)
    assert np.max(np.abs(g_o)) < 1e-15
    assert abs(loss - ent / 2) < 1e-13
    # shifting a node's logits changes nothing; any other logits cost more (Gibbs)
    o2 = o.copy(); o2[:8] += 3.7
    assert abs(mlp.softmax_cross_entropy(o2, t, off)[0] - loss) < 1e-13
    assert mlp.softmax_cross_entropy(g.standard_normal(20), t, off)[0] > loss


def test_adam_constant_gradient_closed_form():
    # with a constant gradient the bias-corrected moments are exactly g and g^2,
    # so every step moves theta by -lr g / (|g| + eps)
    g = np.array([0.5, -2.0, 1e-3, 0.0])
    theta = np.array([1.0, 2.0, 3.0, 4.0])
    m = np.zeros(4); v = np.zeros(4)
    lr, eps = 1e-2, 1e-8
    th = theta.copy()
    for step in range(1, 6):
        th, m, v = mlp.adam_step(th, g, m, v, step, lr, eps=eps)
        expect = theta - step * lr * g / (np.abs(g) + eps)
        assert np.max(np.abs(th - expect)) < 1e-13


def test_weighted_single_draw_probabilities():
    # s = 1: the largest key ln(u)/w' is row i with probability w'_i / sum w'
    o = np.array([0.0, 1.0, -1.0, 2.0, 0.5, -3.0])
    wp = proposal.mixed_weights(o)
    assert abs(np.mean(wp) - 1.0) < 1e-14 and wp.min() > 0.1
    pool = np.arange(100, 106)
    n = 4000
    counts = np.zeros(6)
    for sid in range(n):
        rows, _ = proposal.weighted_select(pool, o, 1, 5, sid)
        counts[rows[0] - 100] += 1
    expect = n * wp / wp.sum()
    chi2 = float(np.sum((counts - expect) ** 2 / expect))
    assert chi2 < 25.0, (counts, expect)     # 5 d.o.f.: P(chi2 > 25) < 2e-4


def test_weighted_select_structure():
    pool = np.arange(50, 90)
    o = np.random.default_rng(2).standard_normal(40)
    rows, keys = proposal.weighted_select(pool, o, 10, 9, 4)
    assert rows.size == 10 and np.unique(rows).size == 10
    kk = keys[rows - 50]
    assert np.all(np.diff(kk) <= 0)
    assert kk[-1] >= np.max(np.delete(keys, rows - 50))
    # equal logits: w' = 1 and the keys are ln(u): the s rows with the largest u
    rows_eq, keys_eq = proposal.weighted_select(pool, np.zeros(40), 10, 9, 4)
    u = np.exp(keys_eq)
    assert list(rows_eq) == list(pool[np.argsort(-u, kind="stable")[:10]])
    all_rows, _ = proposal.weighted_select(pool, o, 100, 9, 4)
    assert sorted(all_rows) == list(pool)


def test_features_closed_form():
    Y = np.array([[3.0, 4.0, 0.0, 0.0]])
    x_c = np.array([1.0, 0.0, 0.0, 0.0])
    proj = np.vstack([np.eye(4), -np.eye(4)])
    rho = 2.0
    # delta = (2, 4, 0, 0), r = sqrt(20), ||y|| = 5
    F = proposal.features(Y, [0], x_c, rho, Kernel(GAUSSIAN, h=1.0), proj)[0]
    assert abs(F[0] - math.sqrt(20) / 2) < 1e-15
    assert abs(F[1] - math.exp(-10.0)) < 1e-18
    assert F[2] == 2.5 and F[3] == 2.0
    assert list(F[4:]) == [1.0, 2.0, 0.0, 0.0, -1.0, -2.0, -0.0, -0.0]
    F = proposal.features(Y, [0], x_c, rho, Kernel(LAPLACE), proj)[0]
    assert abs(F[1] - (4.0 / 20.0)) < 1e-15            # (rho / r)^(d-2) = 4/20
    assert F[3] == 2.0
    F = proposal.features(Y, [0], x_c, rho, Kernel(POLYNOMIAL, h=4.0, c=1.0, p=3), proj)[0]
    assert abs(F[1] - (1.75 / 2.25) ** 3) < 1e-15      # (3/4 + 1)^3 / (5/4 + 1)^3
    assert F[3] == 0.5


def _node_setup(seed=0):
    Y = workloads.gaussian_mixture(4096, 8, 4, seed=seed)
    # the node: the 64 points nearest to the first one, moved to the front
    Y = Y[np.argsort(np.sum((Y - Y[0]) ** 2, axis=1), kind="stable")]
    x_c = Y[:64].mean(axis=0)
    rho = float(np.sqrt(np.max(np.sum((Y[:64] - x_c) ** 2, axis=1))))
    return Y, x_c, rho


def test_proposal_draws_from_the_pool_and_is_prefix_consistent():
    Y, x_c, rho = _node_setup()
    proj = workloads.projections(8, seed=1)
    theta = workloads.mlp_init(seed=2)
    kern = Kernel(GAUSSIAN, h=2.0)
    far = far_field_mask(Y, x_c, rho, 1.0, 0, 64)
    for pool_rows in (0, 600):
        pool = proposal.candidate_pool(far, 3, 17, pool_rows)
        assert pool.size == (far.sum() if pool_rows == 0 else 600)
        big = proposal.propose_from_mask(far, Y, 256, 3, 17, x_c, rho, kern, proj, theta, pool_rows)
        for s in (16, 128):
            rows = proposal.propose_from_mask(far, Y, s, 3, 17, x_c, rho, kern, proj, theta, pool_rows)
            assert rows.size == s and np.unique(rows).size == s
            assert set(rows) <= set(pool) and np.all(far[rows])
            assert list(rows) == list(big[:s])          # keys do not depend on s
    # a far field no larger than s is taken whole
    small = np.zeros_like(far); small[np.flatnonzero(far)[:20]] = True
    rows = proposal.propose_from_mask(small, Y, 32, 3, 17, x_c, rho, kern, proj, theta)
    assert sorted(rows) == list(np.flatnonzero(small))


def test_leverage_targets_of_exact_low_rank_block():
    g = np.random.default_rng(5)
    A = g.standard_normal((300, 5)) @ g.standard_normal((5, 40))
    t, r = proposal.leverage_targets(A, 1e-8)
    assert r == 5 == eps_rank(A, 1e-8)
    Q, _ = np.linalg.qr(A[:, :5])          # the column space of A, by Householder QR
    lev = np.sum(Q * Q, axis=1)
    assert abs(t.sum() - 1.0) < 1e-12
    assert np.max(np.abs(t - lev / 5)) < 1e-12
