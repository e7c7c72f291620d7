"""GPU parity of the single-block path against the FP64 oracle (through the C ABI).

Tolerances (FP64 path, both sides FP64, different summation orders):
* sampled rows, far-field lists: bit-exact (integer work);
* kernel block entries: |K_gpu - K_oracle| <= 1e-13 * max|K| (a few ulps of
  the exp/log/pow of distances formed in another order);
* ID: identical rank; identical skeleton when every consecutive pivot gap
  exceeds 1e-7 relative (else only up to the first near tie); r22 and the
  full-block error e agree to |e_gpu - e_oracle| <= 1e-10 (both already
  relative to ||K||_F, the reading of "match the oracle's ID error to 1e-10").
"""
import numpy as np
import pytest
import torch

import workloads
from oracle import interp as o_interp
from oracle import kernels as o_kernels
from oracle import sampling as o_sampling
from oracle.cpqr import cpqr as o_cpqr
from parity import fp64_error_ok

pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_1409_2802_gb300 import ffc  # noqa: E402

DEV = torch.device("cuda:0")


def cu(a):
    return torch.tensor(np.ascontiguousarray(a), device=DEV)


def okernel(kind, h=1.0, c=1.0, p=3):
    return o_kernels.Kernel(kind, h=h, c=c, p=p), ffc.Kernel(kind, h=h, c=c, p=p)


# ---------------------------------------------------------------- sampling

@pytest.mark.parametrize("s", [1, 37, 256, 2048])
def test_sample_rows_single_block_bit_exact(s):
    X, Y = workloads.single_block(0)
    rows, fc, st = ffc.ffc_sample_rows(cu(Y), s, seed=0, stream_id=0)
    o_rows, o_fc = o_sampling.sample_uniform(Y, s, 0, 0)
    assert np.array_equal(rows.cpu().numpy(), o_rows)
    assert fc == o_fc
    assert st == (ffc.FFC_OK if s <= 2048 else ffc.FFC_E_FARFIELD_TOO_SMALL)


@pytest.mark.parametrize("seed,stream_id,s", [(0, 5, 128), (7, 123, 512), (2**63 + 5, 2**40, 300)])
def test_sample_rows_far_field_and_exclusion_bit_exact(seed, stream_id, s):
    P = workloads.gaussian_mixture(N=20000, d=6, k=4, seed=3)
    node = slice(4000, 6000)
    xc = P[node].mean(axis=0)
    rho = float(np.sqrt(((P[node] - xc) ** 2).sum(1)).max())
    rows, fc, st = ffc.ffc_sample_rows(cu(P), s, seed, stream_id, x_c=cu(xc), radius=rho, xi=1.0,
                                       ex_begin=4000, ex_end=6000)
    o_rows, o_fc = o_sampling.sample_uniform(P, s, seed, stream_id, xc, rho, 1.0, 4000, 6000)
    assert np.array_equal(rows.cpu().numpy(), o_rows)
    assert fc == o_fc


def test_sample_rows_phase_b_and_small_far_field():
    # far field = 60 points of 20,000: phase A runs out and phase B enumerates
    g = np.random.default_rng(0)
    Y = g.random((20000, 3))
    Y[::333][:60] += 10.0
    xc = np.full(3, 0.5)
    for s in (40, 59, 60, 61, 100):
        rows, fc, st = ffc.ffc_sample_rows(cu(Y), s, 9, 2, x_c=cu(xc), radius=5.0)
        o_rows, o_fc = o_sampling.sample_uniform(Y, s, 9, 2, xc, 5.0)
        assert np.array_equal(rows.cpu().numpy(), o_rows), s
        assert fc == o_fc == 60
        assert st == (ffc.FFC_OK if s <= 60 else ffc.FFC_E_FARFIELD_TOO_SMALL)


def test_far_field_list_bit_exact():
    P = workloads.gaussian_mixture(N=30001, d=5, k=4, seed=4)
    xc = P[:1000].mean(0)
    rho = float(np.sqrt(((P[:1000] - xc) ** 2).sum(1)).max())
    idx = ffc.ffc_far_field(cu(P), cu(xc), rho, 1.0, 0, 1000).cpu().numpy()
    mask = o_sampling.far_field_mask(P, xc, rho, 1.0, 0, 1000)
    assert np.array_equal(idx, np.flatnonzero(mask))


def test_sample_rows_empty_cases():
    Y = np.random.default_rng(1).random((100, 2))
    rows, fc, st = ffc.ffc_sample_rows(cu(Y), 0, 0, 0)
    assert rows.numel() == 0 and st == ffc.FFC_OK
    rows, fc, st = ffc.ffc_sample_rows(cu(Y), 10, 0, 0, ex_begin=0, ex_end=100)
    assert rows.numel() == 0 and fc == 0 and st == ffc.FFC_E_FARFIELD_TOO_SMALL


# ---------------------------------------------------------------- kernels

@pytest.mark.parametrize("kind,d,h,s,n", [
    (o_kernels.GAUSSIAN, 4, 1.0, 256, 512),
    (o_kernels.GAUSSIAN, 16, 2.0, 131, 333),     # ragged tiles
    (o_kernels.GAUSSIAN, 70, 3.0, 65, 97),       # several coordinate chunks
    (o_kernels.LAPLACE, 5, 1.0, 100, 200),
    (o_kernels.LAPLACE, 128, 1.0, 64, 150),      # d - 2 = 126: needs the scaling
    (o_kernels.POLYNOMIAL, 6, 6.0, 77, 300),
])
def test_eval_block_matches_oracle(kind, d, h, s, n):
    g = np.random.default_rng(d * 7 + s)
    X = g.standard_normal((n, d))
    Y = g.standard_normal((3 * s, d)) + (2.0 if kind != o_kernels.POLYNOMIAL else 0.0)
    rows = g.choice(3 * s, s, replace=False).astype(np.int64)
    ok, gk = okernel(kind, h=h)
    Ko, ls_o = o_kernels.kernel_block(ok, Y[rows], X)
    Kg, ls_g = ffc.ffc_eval_block(gk, cu(Y), cu(rows), cu(X))
    Kg = Kg.cpu().numpy()
    assert np.max(np.abs(Kg - Ko)) <= 1e-13 * np.max(np.abs(Ko))
    assert ls_g == pytest.approx(ls_o, rel=1e-13, abs=1e-13)


def test_eval_laplace_singular_rejected():
    X = np.zeros((4, 3))
    Y = np.zeros((4, 3))
    with pytest.raises(ffc.FFCError) as e:
        ffc.ffc_eval_block(ffc.Kernel(ffc.LAPLACE), cu(Y), cu(np.arange(4)), cu(X))
    assert e.value.status == ffc.FFC_E_SINGULAR


# ---------------------------------------------------------------- ID

def _determined_pivots(Kblock, r, thr=1e-7, floor=1e-11):
    """How many of the oracle's first r pivots are fixed by the data.

    A pivot is determined when the two largest residual norms differ by more
    than thr (relative) and the largest is above floor * ||K||_F; past the
    numerical rank the residual is rounding noise and any choice is correct.
    """
    A = np.array(Kblock, dtype=np.float64)
    s, n = A.shape
    fro = np.linalg.norm(A)
    selected = np.zeros(n, dtype=bool)
    from oracle.cpqr import householder
    for k in range(min(r, s, n)):
        free = np.flatnonzero(~selected)
        nr = np.sqrt(np.sum(A[k:, free] ** 2, axis=0))
        o = np.sort(nr)[::-1]
        if o[0] <= floor * fro or (o.size > 1 and (o[0] - o[1]) <= thr * o[0]):
            return k
        p = int(free[np.argmax(nr)])
        v, tau, beta = householder(A[k:, p])
        rest = free[free != p]
        A[k:, rest] -= tau * np.outer(v, v @ A[k:, rest])
        selected[p] = True
    return min(r, s, n)


def _check_id(Ko, r_max, tol, ok=None, Y=None, X=None, gk=None):
    n = Ko.shape[1]
    ref = o_interp.interpolative_decomposition(Ko, r_max, tol)
    Kst = cu(Ko.T.copy())                       # column-major storage: (n, s) row-major
    skel, T, r, r22, st = ffc.ffc_id(Kst, r_max, tol)
    skel, T = skel.cpu().numpy().astype(np.int64), T.cpu().numpy()
    assert r == ref["rank"]
    assert abs(r22 - ref["r22_rel"]) <= 1e-10
    k_det = _determined_pivots(Ko, r)
    assert np.array_equal(skel[:k_det], ref["skel_perm"][:k_det])
    if k_det == r:
        assert np.array_equal(skel, ref["skel_perm"])
        # T itself is only as well determined as R11 is conditioned (entries
        # differ by ~ cond(R11) * eps); what the ID delivers, C P, must agree
        # to rounding: ||K(:,J) (P_gpu - P_oracle)||_F / ||K||_F
        Pg = o_interp.assemble_P(skel, T, n)
        Po = o_interp.assemble_P(ref["skel_perm"], ref["T"], n)
        J = skel[:r]
        diff = np.linalg.norm(Ko[:, J] @ (Pg - Po)) / max(np.linalg.norm(Ko), 1e-300)
        assert diff <= 1e-12, diff
    # the GPU ID reproduces the block to its own r22
    assert o_interp.reconstruction_error(Ko, skel, T) == pytest.approx(r22, rel=1e-6, abs=1e-14)
    if ok is not None:
        e_g = ffc.ffc_id_error(gk, cu(Y), cu(X), cu(skel.astype(np.int32)), cu(T), r)
        e_o = o_interp.full_block_error(ok, Y, X, ref["skel_perm"], ref["T"])
        assert fp64_error_ok(e_g, e_o), (e_g, e_o, abs(e_g - e_o))
    return r, st


def test_id_single_block_rank_64_and_tol():
    X, Y = workloads.single_block(0)
    ok, gk = okernel(o_kernels.GAUSSIAN, h=1.0)
    rows, _ = o_sampling.sample_uniform(Y, 256, 0, 0)
    Ko, _ = o_kernels.kernel_block(ok, Y[rows], X)
    r, st = _check_id(Ko, 64, 0.0, ok, Y, X, gk)
    assert r == 64 and st == ffc.FFC_OK
    r, st = _check_id(Ko, 256, 1e-6, ok, Y, X, gk)
    assert 64 < r < 128 and st == ffc.FFC_OK


@pytest.mark.parametrize("s,n,r_max,tol,seed", [
    (1, 5, 3, 0.0, 0), (7, 3, 5, 0.0, 1), (64, 64, 64, 0.0, 2), (200, 333, 50, 0.0, 3),
    (300, 1000, 150, 1e-9, 4), (2048, 700, 1024, 1e-12, 5), (33, 2000, 33, 0.0, 6),
])
def test_id_shapes_against_oracle(s, n, r_max, tol, seed):
    K = workloads.random_matrix(s, n, seed=seed, decay=0.85) + 1e-14 * workloads.random_matrix(s, n, seed=seed + 1)
    _check_id(K, r_max, tol)


def test_id_rank_zero_and_zero_columns():
    K = workloads.random_matrix(40, 30, seed=8, decay=0.5)
    K[:, 5] = 0.0
    K[:, 17] = 0.0
    _check_id(K, 0, 0.0)
    r, _ = _check_id(K, 30, 0.0)
    assert r == 28                      # the two zero columns are never selected
    skel, T, r, r22, st = ffc.ffc_id(cu(np.zeros((30, 40))), 10, 1e-6)
    assert r == 0 and r22 == 0.0


def test_id_tol_not_reached_is_soft():
    K = workloads.random_matrix(50, 60, seed=9)
    skel, T, r, r22, st = ffc.ffc_id(cu(K.T.copy()), 10, 1e-12)
    assert r == 10 and st == ffc.FFC_E_TOL_NOT_REACHED and r22 > 1e-12


@pytest.mark.parametrize("kind,d,h", [(o_kernels.LAPLACE, 5, 1.0), (o_kernels.POLYNOMIAL, 4, 4.0)])
def test_id_error_other_kernels(kind, d, h):
    g = np.random.default_rng(11)
    X = g.standard_normal((300, d))
    Y = g.standard_normal((900, d)) + 4.0
    ok, gk = okernel(kind, h=h)
    rows, _ = o_sampling.sample_uniform(Y, 128, 3, 1)
    Ko, _ = o_kernels.kernel_block(ok, Y[rows], X)
    _check_id(Ko, 40, 0.0, ok, Y, X, gk)


def test_id_error_of_oracle_id_bit_close():
    """ffc_id_error on the oracle's own ID equals the oracle's error."""
    X, Y = workloads.single_block(0)
    ok, gk = okernel(o_kernels.GAUSSIAN, h=1.0)
    rows, _ = o_sampling.sample_uniform(Y, 256, 0, 0)
    Ko, _ = o_kernels.kernel_block(ok, Y[rows], X)
    for r in (0, 1, 64, 200, 256):
        ref = o_interp.interpolative_decomposition(Ko, r)
        e_o = o_interp.full_block_error(ok, Y, X, ref["skel_perm"], ref["T"])
        e_g = ffc.ffc_id_error(gk, cu(Y), cu(X), cu(ref["skel_perm"].astype(np.int32)), cu(ref["T"]), ref["rank"])
        assert abs(e_g - e_o) <= 1e-12 * max(e_o, 1e-3), (r, e_g, e_o)
