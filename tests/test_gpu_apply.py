"""GPU parity of the outgoing representation (§2.1.3): skeleton charges q~ = P q,
potentials C q~ and K q, and the potential at every point of a compressed tree,
against the oracle (the oracle's own IDs; the GPU's IDs equal them to rounding
by the tree parity tests).

Tolerances. Charges and single-block potentials are sums of at most a few
thousand FP64 products in another order than the oracle's: 1e-12 relative to
the largest magnitude. Tree potentials additionally carry the difference
between the two sides' IDs (T agrees to about cond(R11) eps): 1e-9 relative.
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

pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_1409_2802_gb300 import ffc  # noqa: E402

DEV = torch.device("cuda:0")


def cu(a):
    return torch.tensor(np.ascontiguousarray(a), device=DEV)


def _kernels(d):
    return [(o_kernels.Kernel(o_kernels.GAUSSIAN, h=1.0), ffc.Kernel(ffc.GAUSSIAN, h=1.0)),
            (o_kernels.Kernel(o_kernels.LAPLACE), ffc.Kernel(ffc.LAPLACE)),
            (o_kernels.Kernel(o_kernels.POLYNOMIAL, h=float(d), c=1.0, p=3),
             ffc.Kernel(ffc.POLYNOMIAL, h=float(d), c=1.0, p=3))]


@pytest.mark.parametrize("r_max", [0, 1, 37, 300])
def test_skeleton_charges_match_oracle(r_max):
    K = workloads.random_matrix(400, 300, seed=r_max + 3, decay=0.9)
    ref = o_interp.interpolative_decomposition(K, r_max)
    skel, T, r = ref["skel_perm"], ref["T"], ref["rank"]
    q = np.random.default_rng(r_max).standard_normal((300, 3))
    qt_o = np.stack([o_apply.skeleton_charges(skel, T, q[:, j]) for j in range(3)], axis=1)
    qt_g = ffc.ffc_skeleton_charges(cu(skel.astype(np.int32)), cu(T), cu(q)).cpu().numpy()
    assert qt_g.shape == (r, 3)
    if r:
        assert np.max(np.abs(qt_g - qt_o)) <= 1e-12 * np.max(np.abs(qt_o))


@pytest.mark.parametrize("which", [0, 1, 2])
def test_potentials_match_oracle(which):
    X, Y = workloads.single_block(0)
    Y = Y.copy()
    ok, gk = _kernels(4)[which]
    rows = np.sort(np.random.default_rng(1).choice(len(Y), 333, replace=False))
    q = np.random.default_rng(2).standard_normal(len(X))
    Ko, ls = o_kernels.kernel_block(ok, Y[rows], X)
    # the direct sum, on the oracle's scale of the block
    u_o, _ = o_apply.direct_potential(ok, Y[rows], X, q)
    u_g = ffc.ffc_potential(gk, cu(Y), cu(X), cu(q), rows=cu(rows), log_scale=ls).cpu().numpy()
    assert np.max(np.abs(u_g - u_o)) <= 1e-12 * np.max(np.abs(u_o))
    # the representation's potential C q~ with the oracle's ID of the sampled block
    ref = o_interp.interpolative_decomposition(Ko, 40)
    skel, T, r = ref["skel_perm"], ref["T"], ref["rank"]
    qt = o_apply.skeleton_charges(skel, T, q)
    ut_o, _ = o_apply.id_potential(ok, Y[rows], X, skel, r, qt)
    ut_g = ffc.ffc_potential(gk, cu(Y), cu(X), cu(qt), rows=cu(rows), cols=cu(skel[:r].astype(np.int32)),
                             log_scale=ls).cpu().numpy()
    assert np.max(np.abs(ut_g - ut_o)) <= 1e-12 * np.max(np.abs(ut_o))


def _tree_case(N=4096, d=4, leaf=256, seed=1):
    P = workloads.gaussian_mixture(N=N, d=d, k=4, seed=seed)
    t_o = o_tree.build_tree(P, leaf)
    t_g = ffc.ffc_build_tree(cu(P), leaf)
    return P[t_o.perm], t_o, t_g


@pytest.mark.parametrize("which", [0, 1, 2])
def test_tree_apply_matches_oracle(which):
    Pp, t_o, t_g = _tree_case()
    ok, gk = _kernels(4)[which]
    if which == 2:        # a cubic in d = 4 has exact rank C(7, 3) = 35
        ok, gk = o_kernels.Kernel(o_kernels.POLYNOMIAL, h=4.0, c=1.0, p=3), ffc.Kernel(ffc.POLYNOMIAL, h=4.0, c=1.0, p=3)
    s0, s_max, tol = 32, 512, 1e-6
    res = ffc.ffc_compress_tree(cu(Pp), t_g, gk, tol=tol, s0=s0, s_max=s_max)
    nodes = [i for i in range(t_o.n_nodes) if t_o.level[i] >= 2]
    refs = {nd: o_compress.compress_node(Pp, t_o, nd, ok, tol, 0, s0, s_max) for nd in nodes}
    ids = {nd: (rf.skel_perm, rf.T, rf.rank) for nd, rf in refs.items() if rf.status in (0, 7)}
    q = np.random.default_rng(3).standard_normal(len(Pp))
    u_s_o = o_apply.tree_potential(ok, Pp, t_o, q, ids, mode="skeleton")
    u_d_o = o_apply.tree_potential(ok, Pp, t_o, q, mode="direct")
    u_s_g, qt = ffc.ffc_tree_apply(cu(Pp), t_g, res, cu(q), mode=ffc.APPLY_SKELETON, s_max=s_max)
    u_d_g, _ = ffc.ffc_tree_apply(cu(Pp), t_g, res, cu(q), mode=ffc.APPLY_DIRECT, s_max=s_max)
    u_s_g, u_d_g = u_s_g.cpu().numpy(), u_d_g.cpu().numpy()
    scale = np.max(np.abs(u_d_o))
    assert np.max(np.abs(u_d_g - u_d_o)) <= 1e-12 * scale
    assert np.max(np.abs(u_s_g - u_s_o)) <= 1e-9 * scale
    # the direct mode with the near field is the all-pairs sum without self
    u_all = o_apply.direct_sum_without_self(ok, Pp, q)
    assert np.max(np.abs(u_d_g - u_all)) <= 1e-12 * np.max(np.abs(u_all))
    # the representation's error against the exact far field, as the oracle sees it
    e_g = np.linalg.norm(u_s_g - u_d_g) / np.linalg.norm(u_d_g)
    e_o = np.linalg.norm(u_s_o - u_d_o) / np.linalg.norm(u_d_o)
    print(f"kernel {which}: relative error of the tree evaluation {e_g:.3e} (oracle {e_o:.3e})")
    assert abs(e_g - e_o) <= 1e-9 + 1e-6 * e_o
    # skeleton charges of every compressed node against the oracle's q~
    h = ffc.tree_result_to_host(res)
    qt = qt.cpu().numpy()
    for i, nd in enumerate(h["node"]):
        rf = refs[int(nd)]
        if rf.status not in (0, 7) or rf.rank == 0 or not np.array_equal(
                h["skel"][h["skel_off"][i]: h["skel_off"][i] + rf.rank], rf.skel_perm[:rf.rank]):
            continue
        bg, n = int(t_o.begin[nd]), int(t_o.count[nd])
        qt_o = o_apply.skeleton_charges(rf.skel_perm, rf.T, q[bg:bg + n])
        assert np.max(np.abs(qt[i, :rf.rank] - qt_o)) <= 1e-9 * max(np.max(np.abs(qt_o)), 1.0), int(nd)


def test_tree_apply_full_size_d16_sampled_targets():
    """The benchmark tree (N = 65,536, d = 16, Gaussian h = 2), far field only: the direct mode at 256
    seeded targets against the oracle's (the interaction lists and sums, exact to rounding); the
    skeleton mode runs at full size and its relative error against the direct mode is reported."""
    P = workloads.gaussian_mixture(N=65536, d=16, k=8, seed=0)
    t_o = o_tree.build_tree(P, 256)
    t_g = ffc.ffc_build_tree(cu(P), 256)
    Pp = P[t_o.perm]
    ok, gk = o_kernels.Kernel(o_kernels.GAUSSIAN, h=2.0), ffc.Kernel(ffc.GAUSSIAN, h=2.0)
    res = ffc.ffc_compress_tree(cu(Pp), t_g, gk, tol=1e-6, s0=128, s_max=2048)
    q = np.random.default_rng(5).standard_normal(len(Pp))
    u_d, _ = ffc.ffc_tree_apply(cu(Pp), t_g, res, cu(q), mode=ffc.APPLY_DIRECT, near_field=False)
    u_s, _ = ffc.ffc_tree_apply(cu(Pp), t_g, res, cu(q), mode=ffc.APPLY_SKELETON, near_field=False)
    u_d, u_s = u_d.cpu().numpy(), u_s.cpu().numpy()
    sub = np.sort(np.random.default_rng(6).choice(len(Pp), 256, replace=False))
    u_d_o = o_apply.tree_potential(ok, Pp, t_o, q, mode="direct", near=False, targets=sub)
    assert np.max(np.abs(u_d[sub] - u_d_o)) <= 1e-12 * np.max(np.abs(u_d_o))
    # uniformly sampled rows leave most of these blocks' full-block ID errors near 1 (the sampled
    # rows miss the far field's dominant rows), and the evaluation inherits that: reported, bounded by
    # the sum of the far fields' magnitudes
    e = np.linalg.norm(u_s - u_d) / np.linalg.norm(u_d)
    print(f"N=65536: relative far-field error of the skeleton evaluation {e:.3e}")
    assert np.all(np.isfinite(u_s)) and e < 2.0
