"""Pins for the oracle's kernels, pivoted QR and interpolative decomposition.

Each check is fixed by the paper or by mathematics, not by the oracle itself:
closed-form kernel values (§4.2-§4.4), Silverman's bandwidth (Tables 2 and 4),
LAPACK's pivoted QR (geqp3) as the textbook routine, the ID definition
(P contains I_r; §2.1.3), the identity ||K' - K'(:,J)P||_F = ||R22||_F, the
optimality of the truncated SVD (§2.1.3), the ID error bound (§2.1.3), the
exact rank C(d+p, p) of the degree-p polynomial kernel, the h -> infinity
limit of the Gaussian (§4.2.1) and the problem case of §3.
"""
import json
import math
import os

import numpy as np
import pytest
import scipy.linalg as sl

import workloads
from oracle import cpqr as cq
from oracle import interp, kernels, spectral
from oracle.kernels import GAUSSIAN, LAPLACE, POLYNOMIAL, Kernel

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_silverman_matches_tables_2_and_4():
    with open(os.path.join(GOLDEN, "silverman_bandwidth.json")) as f:
        g = json.load(f)
    for c in g["cases"]:
        assert round(kernels.silverman_bandwidth(c["d"], c["N"]), 4) == pytest.approx(c["h_S"], abs=1e-12)


def test_kernel_closed_form_values():
    y, x = np.array([0.0, 0.0]), np.array([1.0, 1.0])
    assert kernels.kernel_value(Kernel(GAUSSIAN, h=1.0), y, x) == pytest.approx(math.exp(-1.0), rel=1e-15)
    y4, x4 = np.zeros(4), np.array([2.0, 0, 0, 0])
    assert kernels.kernel_value(Kernel(LAPLACE), y4, x4) == pytest.approx(0.25, rel=1e-15)
    y3, x3 = np.zeros(3), np.array([0, 0, 2.0])
    assert kernels.kernel_value(Kernel(LAPLACE), y3, x3) == pytest.approx(0.5, rel=1e-15)
    assert kernels.kernel_value(Kernel(POLYNOMIAL, h=2.0, c=1.0, p=3), np.array([1.0, 2.0]),
                                np.array([3.0, 4.0])) == pytest.approx(6.5 ** 3, rel=1e-15)


@pytest.mark.parametrize("kind,d", [(GAUSSIAN, 4), (LAPLACE, 5), (LAPLACE, 16), (POLYNOMIAL, 6)])
def test_kernel_block_matches_scalar_formula(kind, d):
    g = np.random.default_rng(d)
    Y = g.random((7, d)) + 2.0
    X = g.random((5, d))
    k = Kernel(kind, h=0.7 if kind == GAUSSIAN else float(d))
    K, log_scale = kernels.kernel_block(k, Y, X)
    ref = np.array([[kernels.kernel_value(k, y, x) for x in X] for y in Y])
    np.testing.assert_allclose(K * math.exp(log_scale), ref, rtol=1e-13)
    if kind == LAPLACE:
        assert K.max() == pytest.approx(1.0, rel=1e-15)


def test_laplace_rejects_singular_and_d2():
    with pytest.raises(kernels.KernelDomainError):
        kernels.kernel_block(Kernel(LAPLACE), np.zeros((1, 3)), np.zeros((1, 3)))
    with pytest.raises(kernels.KernelDomainError):
        kernels.kernel_block(Kernel(LAPLACE), np.ones((1, 2)), np.zeros((1, 2)))


def test_householder_reflects_onto_e1():
    x = np.array([3.0, 4.0, 12.0])
    v, tau, beta = cq.householder(x)
    Hx = x - tau * v * (v @ x)
    np.testing.assert_allclose(Hx, [beta, 0, 0], atol=1e-14)
    assert beta == pytest.approx(-13.0)          # dlarfg sign: -sign(alpha)*||x||
    v, tau, beta = cq.householder(np.array([-2.0, 0.0]))
    assert tau == 0.0 and beta == -2.0


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_cpqr_matches_lapack_geqp3(seed):
    K = workloads.random_matrix(60, 40, seed=seed, decay=0.7)
    K = K * np.linspace(1.0, 3.0, 40)[None, :]          # spread the column norms
    qr = cq.cpqr(K, 25)
    Q, R, piv = sl.qr(K, pivoting=True, mode="economic")
    assert np.array_equal(qr["piv"], piv[:25])
    res = interp.interpolative_decomposition(K, 25)
    r = 25
    R11 = np.array([[qr["A"][i, qr["piv"][k]] if i <= k else 0.0 for k in range(r)] for i in range(r)])
    np.testing.assert_allclose(np.abs(np.diag(R11)), np.abs(np.diag(R)[:r]), rtol=1e-12)
    np.testing.assert_allclose(qr["r22"], np.linalg.norm(R[r:, r:]), rtol=1e-10)
    assert res["rank"] == r


def test_back_substitution_matches_triangular_solver():
    g = np.random.default_rng(0)
    R = np.triu(g.standard_normal((12, 12))) + 5 * np.eye(12)
    B = g.standard_normal((12, 7))
    np.testing.assert_allclose(interp.back_substitution(R, B), sl.solve_triangular(R, B), rtol=1e-12)


def _c1_block():
    X, Y = workloads.single_block(0)
    from oracle.sampling import sample_uniform
    rows, _ = sample_uniform(Y, 256, 0, 0)
    K, _ = kernels.kernel_block(Kernel(GAUSSIAN, h=1.0), Y[rows], X)
    return X, Y, K


def test_id_definition_and_r22_identity():
    _, _, K = _c1_block()
    res = interp.interpolative_decomposition(K, 64)
    P = interp.assemble_P(res["skel_perm"], res["T"], K.shape[1])
    J = res["skel_perm"][:64]
    assert np.array_equal(P[:, J], np.eye(64))                 # P contains I_r exactly
    err = np.linalg.norm(K - K[:, J] @ P) / np.linalg.norm(K)
    assert err == pytest.approx(res["r22_rel"], rel=1e-8)
    assert interp.reconstruction_error(K, res["skel_perm"], res["T"]) == pytest.approx(err, rel=1e-8)


def test_r22_monotone_and_bounded_below_by_svd():
    g = np.random.default_rng(3)
    K = workloads.random_matrix(40, 30, seed=3, decay=0.6) + 1e-9 * g.standard_normal((40, 30))
    prev = np.inf
    for r in range(0, 21):
        res = interp.interpolative_decomposition(K, r)
        assert res["r22_rel"] <= prev * (1 + 1e-12)
        prev = res["r22_rel"]
        e_svd = spectral.svd_frobenius_error(K, r)
        assert res["r22_rel"] >= e_svd * (1 - 1e-10)
        # ID theorem: ||K - CP||_2 <= sqrt(1 + n r (n - r)) sigma_{r+1}
        P = interp.assemble_P(res["skel_perm"], res["T"], 30)
        J = res["skel_perm"][:r]
        sv = spectral.singular_values(K)
        e2 = np.linalg.norm(K - K[:, J] @ P, 2)
        assert e2 <= math.sqrt(1 + 30 * r * (30 - r)) * sv[r] * (1 + 1e-8)


def test_tol_mode_picks_smallest_rank():
    _, _, K = _c1_block()
    res = interp.interpolative_decomposition(K, 256, tol=1e-6)
    r = res["rank"]
    assert res["r22_rel"] <= 1e-6
    assert interp.interpolative_decomposition(K, r - 1)["r22_rel"] > 1e-6


def test_polynomial_kernel_exact_rank():
    # (x.y/h + 1)^3 in d = 4 spans C(4+3, 3) = 35 monomials: rank <= 35
    g = np.random.default_rng(5)
    X = g.standard_normal((200, 4))
    Y = g.standard_normal((300, 4)) + 3.0
    k = Kernel(POLYNOMIAL, h=4.0, c=1.0, p=3)
    K, _ = kernels.kernel_block(k, Y, X)
    assert math.comb(4 + 3, 3) == 35
    e35 = interp.interpolative_decomposition(K, 35)
    e34 = interp.interpolative_decomposition(K, 34)
    assert interp.reconstruction_error(K, e35["skel_perm"], e35["T"]) < 1e-10
    assert interp.reconstruction_error(K, e34["skel_perm"], e34["T"]) > 1e-8


def test_gaussian_large_bandwidth_is_rank_one():
    X, Y = workloads.single_block(1, n=100, m=300)
    K, _ = kernels.kernel_block(Kernel(GAUSSIAN, h=1e8), Y, X)
    assert interp.interpolative_decomposition(K, 50, tol=1e-6)["rank"] == 1


def test_problem_case_of_section_3():
    # row 0 = v1, rows 1.. = v2 (v1 orthogonal to v2): rank 2, coherence 1
    m, n = 400, 30
    v1 = np.zeros(n); v1[0] = 1.0
    v2 = np.zeros(n); v2[1:] = 1.0 / math.sqrt(n - 1)
    K = np.vstack([v1[None, :], np.tile(v2, (m - 1, 1))])
    lev = spectral.row_leverage_scores(K, 2)
    assert lev[0] == pytest.approx(1.0, abs=1e-12)
    assert spectral.coherence(K, 2) == pytest.approx(1.0, abs=1e-12)
    # a sample without row 0 loses v1: row 0 is not reproduced at all
    rows = np.arange(1, 41)
    res = interp.interpolative_decomposition(K[rows], 2)
    P = interp.assemble_P(res["skel_perm"], res["T"], n)
    E = K - K[:, res["skel_perm"][:2]] @ P
    assert np.linalg.norm(E[0]) == pytest.approx(1.0, rel=1e-12)
    assert interp.reconstruction_error(K, res["skel_perm"], res["T"]) == pytest.approx(1 / math.sqrt(m), rel=1e-12)
    # a sample holding row 0 (what leverage sampling picks first) is exact
    rows = np.arange(0, 40)
    res = interp.interpolative_decomposition(K[rows], 2)
    assert interp.reconstruction_error(K, res["skel_perm"], res["T"]) < 1e-12
