"""GPU parity of the learned proposal (features, network forward/backward, Adam,
weighted draw, proposal) and of the exact leverage scores, against the oracle;
GPU training and what the trained network gains over uniform sampling."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import workloads
from oracle import mlp as omlp
from oracle import proposal as oprop
from oracle.kernels import GAUSSIAN, LAPLACE, POLYNOMIAL, Kernel
from oracle.sampling import far_field_mask
from oracle.spectral import singular_values

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ffc():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1409_2802_gb300 import ffc as _ffc
    return _ffc


DEV = "cuda"


def _t(a, dtype=None):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dtype).to(DEV)


def _node(seed=0, N=4096, d=16, n=128, gen="mixture"):
    """Points sorted by distance to the first one; the node is the first n."""
    if gen == "mixture":
        Y = workloads.gaussian_mixture(N, d, 4, seed=seed)
    else:
        Y = workloads.low_intrinsic(N, 6, d, seed=seed).astype(np.float64)
    Y = Y[np.argsort(np.sum((Y - Y[0]) ** 2, axis=1), kind="stable")]
    x_c = Y[:n].mean(axis=0)
    rho = float(np.sqrt(np.max(np.sum((Y[:n] - x_c) ** 2, axis=1))))
    return np.ascontiguousarray(Y), x_c, rho


def _params(seed):
    g = np.random.default_rng(seed)
    th = workloads.mlp_init(seed).astype(np.float64) + 0.05 * g.standard_normal(workloads.MLP_N_PARAMS)
    return th.astype(np.float32)


@pytest.mark.parametrize("kind", [GAUSSIAN, LAPLACE, POLYNOMIAL])
@pytest.mark.parametrize("pts", ["f64", "f32"])
def test_features_match_oracle(ffc, kind, pts):
    d = 16 if pts == "f64" else 48
    Y, x_c, rho = _node(seed=1, d=d, gen="mixture" if pts == "f64" else "low")
    if pts == "f32":
        Y = Y.astype(np.float32)
    kern = {GAUSSIAN: Kernel(GAUSSIAN, h=2.0), LAPLACE: Kernel(LAPLACE), POLYNOMIAL: Kernel(POLYNOMIAL, h=float(d))}[kind]
    proj = workloads.projections(d, seed=2)
    far = np.flatnonzero(far_field_mask(Y, x_c, rho, 1.0, 0, 128))
    rows = far[:1001]                       # a ragged count
    Fo = oprop.features(Y, rows, x_c, rho, kern, proj)
    Fg = ffc.ffc_features(ffc.Kernel(kern.kind, kern.h, kern.c, kern.p), _t(Y), _t(rows), _t(x_c), rho,
                          _t(proj)).cpu().numpy()
    assert Fg.shape == (rows.size, 12)
    # O(d) sums in FP32 on coordinates rounded to FP32: relative 2e-5 on the
    # norms; the kernel feature amplifies the distance's error by
    # r^2 / h^2 (Gaussian) or d - 2 (Laplace); projections are held to an
    # absolute error scaled by the magnitudes that enter them
    for f in (0, 2, 3):
        np.testing.assert_allclose(Fg[:, f], Fo[:, f], rtol=2e-5)
    amp = {GAUSSIAN: Fo[:, 0] ** 2 * (rho / 2.0) ** 2, LAPLACE: np.full(rows.size, d - 2.0),
           POLYNOMIAL: np.full(rows.size, 3.0 * d)}[kind]
    assert np.all(np.abs(Fg[:, 1] - Fo[:, 1]) <= 4e-6 * (1.0 + amp) * np.abs(Fo[:, 1]) + 1e-37)
    scale = Fo[:, 0] + Fo[:, 2] + np.linalg.norm(x_c) / rho
    assert np.all(np.abs(Fg[:, 4:] - Fo[:, 4:]) <= 2e-5 * scale[:, None])


def _forward_error_bound(th, F):
    """Bound on |o_gpu - o_oracle| of the inference pass: FP32 sums and GELUs.

    Every FP32 operation, the two-plane FP16 form of h1 (2^-22 relative) and the
    GELU approximation (0.75e-7 |z|) perturb a layer's values by at most about
    c u times the sum of the magnitudes that enter it (u = 2^-24; c = 64 covers
    the 12- and 128-term sums and the GELU); the perturbation of z1 passes
    through |GELU'| <= 1.13 and |W2|, that of z2 through |w3|."""
    p = omlp.unpack(omlp.half_weights(th))
    X = F.astype(np.float64)
    o, (_, z1, h1, z2, h2) = omlp.forward(omlp.half_weights(th), X)
    u = 2.0 ** -24
    c = 64.0
    dz1 = c * u * (np.abs(X) @ np.abs(p["W1"]).T + np.abs(p["b1"]) + np.abs(z1))
    dh1 = 1.13 * dz1 + c * u * (np.abs(h1) + np.abs(z1))
    dz2 = dh1 @ np.abs(p["W2"]).T + c * u * (np.abs(h1) @ np.abs(p["W2"]).T + np.abs(p["b2"]))
    dh2 = 1.13 * dz2 + c * u * (np.abs(h2) + np.abs(z2))
    do = dh2 @ np.abs(p["w3"]) + c * u * (np.abs(h2) @ np.abs(p["w3"]) + abs(p["b3"][0]))
    return o, do


@pytest.mark.parametrize("R", [1000, 1, 128, 50000, 63, 65])
def test_forward_matches_oracle(ffc, R):
    """Inference forward (tensor-core product of the FP16 weights and the FP32
    activations in two FP16 planes) against the oracle's FP64 pass."""
    th = _params(3)
    F = (1.5 * np.random.default_rng(4).standard_normal((R, 12))).astype(np.float32)   # ragged tails
    og = ffc.ffc_mlp_forward(_t(th), _t(F)).cpu().numpy()
    oo, bound = _forward_error_bound(th, F)
    err = np.abs(og - oo)
    print(f"R={R}: max |o_gpu - o_oracle| {err.max():.3e}, max ratio to the bound {np.max(err / bound):.3f}")
    assert np.all(err <= bound)


def test_loss_grad_match_oracle_and_are_deterministic(ffc):
    th = _params(5)
    g = np.random.default_rng(6)
    sizes = [100, 1, 257, 64]
    off = np.concatenate([[0], np.cumsum(sizes)])
    R = int(off[-1])
    F = (1.2 * g.standard_normal((R, 12))).astype(np.float32)
    t = g.random(R) ** 3 * 5.0                  # unnormalised targets
    lo, go = omlp.loss_and_grad(th, F.astype(np.float64), t, off, half=True)
    loss, grad = ffc.ffc_mlp_loss_grad(_t(th), _t(F), _t(t), _t(off, torch.int64))
    gg = grad.cpu().numpy().astype(np.float64)
    assert abs(loss - lo) <= 1e-5 * abs(lo)
    # b3's gradient sum_i (p_i - q_i) is zero in exact arithmetic (softmax is
    # shift invariant), so every group is held to a share of the whole gradient
    gnorm = np.linalg.norm(go)
    for name, (o, shape) in omlp.LAYOUT.items():
        sz = int(np.prod(shape))
        a, b = gg[o:o + sz], go[o:o + sz]
        assert np.linalg.norm(a - b) <= 1e-4 * np.linalg.norm(b) + 1e-6 * gnorm, name
    loss2, grad2 = ffc.ffc_mlp_loss_grad(_t(th), _t(F), _t(t), _t(off, torch.int64))
    assert loss2 == loss and torch.equal(grad, grad2)


def test_adam_matches_oracle(ffc):
    g = np.random.default_rng(7)
    n = workloads.MLP_N_PARAMS
    th = g.standard_normal(n).astype(np.float32)
    gr = (g.standard_normal(n) * 1e-2).astype(np.float32)
    m = (g.standard_normal(n) * 1e-2).astype(np.float32)
    v = (g.random(n) * 1e-4).astype(np.float32)
    to, mo, vo = omlp.adam_step(th, gr, m, v, 3, 1e-3)
    tg, mg, vg = _t(th), _t(m), _t(v)
    ffc.ffc_adam_step(tg, _t(gr), mg, vg, 3, 1e-3)
    np.testing.assert_allclose(tg.cpu().numpy(), to, rtol=2e-7, atol=1e-9)
    np.testing.assert_allclose(mg.cpu().numpy(), mo, rtol=2e-7, atol=1e-12)
    np.testing.assert_allclose(vg.cpu().numpy(), vo, rtol=2e-7, atol=1e-14)


@pytest.mark.parametrize("P,s", [(5000, 700), (16384, 2048), (300, 1), (40, 40), (40, 100), (1, 5),
                                 (50000, 2048), (40000, 8192), (16385, 7)])
def test_weighted_draw_matches_oracle(ffc, P, s):
    g = np.random.default_rng(P + s)
    pool = g.choice(10 ** 6, size=P, replace=False).astype(np.int64)
    logits = (2.0 * g.standard_normal(P)).astype(np.float32)
    rows_o, keys = oprop.weighted_select(pool, logits.astype(np.float64), s, 11, 42)
    rows_g = ffc.ffc_sample_weighted(_t(pool), _t(logits), s, 11, 42).cpu().numpy()
    if not np.array_equal(rows_g, rows_o):
        # only an exact tie in FP64 keys may reorder; there must be none in a random pool
        srt = np.sort(keys)[::-1]
        assert np.min(np.abs(np.diff(srt[:min(s, P) + 1]))) < 1e-14 * np.abs(srt[0]), "selection differs"


def test_weighted_draw_with_clustered_keys_is_the_exact_selection(ffc):
    """Logits that put most keys ln(u_i) / w'_i within about 1e-7 of one value: the FP32 pre-selection's
    window (about 5e-5 relative around the cut) then holds far more rows than the shared-memory sort, so
    the draw takes the exact radix selection over FP64 keys. It must be the oracle's selection, and in
    the oracle's key order, wherever the FP64 keys differ by more than their rounding (1e-15)."""
    from oracle.philox import DOMAIN_WEIGHTED_KEYS, draws, to_unit_double
    P, s, seed, stream_id = 40000, 8192, 5, 17
    L = -np.log(to_unit_double(draws(seed, stream_id, DOMAIN_WEIGHTED_KEYS, 0, P)))
    # w'_i = 0.9 r_i + 0.1 with r_i = w_i / mean(w); r_i = (L_i / c - 0.1) / 0.9 makes key_i = -c, and
    # mean(r) = 1 fixes c (bisection; rows with L_i < 0.1 c take r = 1e-3 and rank above the cluster)
    def mean_r(c):
        return np.mean(np.maximum((L / c - 0.1) / 0.9, 1e-3))
    lo_c, hi_c = 0.25 * L.mean(), 4.0 * L.mean()
    for _ in range(100):
        mid = 0.5 * (lo_c + hi_c)
        lo_c, hi_c = (mid, hi_c) if mean_r(mid) > 1.0 else (lo_c, mid)
    r = np.maximum((L / lo_c - 0.1) / 0.9, 1e-3)
    logits = np.log(r).astype(np.float32)
    pool = np.arange(P, dtype=np.int64) * 3 + 1
    rows_o, keys = oprop.weighted_select(pool, logits.astype(np.float64), s, seed, stream_id)
    cut = np.sort(keys)[::-1][s - 1]
    assert np.sum(np.abs(keys - cut) <= 5e-5 * abs(cut)) > 16384   # the window overflows the sort
    rows_g = ffc.ffc_sample_weighted(_t(pool), _t(logits), s, seed, stream_id).cpu().numpy()
    assert rows_g.size == s and np.unique(rows_g).size == s
    kg = keys[(rows_g - 1) // 3]
    tol = 1e-15 * np.abs(keys).max()
    assert np.all(np.diff(kg) <= tol), "not in decreasing key order"
    rest = np.setdiff1d(np.arange(P), (rows_g - 1) // 3)
    assert np.max(keys[rest]) <= kg.min() + tol, "a better row was left out"
    print(f"identical to the oracle: {np.array_equal(rows_g, rows_o)}")


@pytest.mark.parametrize("pool_rows", [0, 3000])
def test_proposal_is_a_valid_draw_from_the_oracle_pool(ffc, pool_rows):
    Y, x_c, rho = _node(seed=2, N=8192)
    kern = Kernel(GAUSSIAN, h=2.0)
    proj = workloads.projections(16, seed=3)
    th = _params(8)
    far = far_field_mask(Y, x_c, rho, 1.0, 0, 128)
    prev = None
    for s in (64, 200):
        rows_g, fc, st = ffc.ffc_propose_rows(ffc.Kernel(GAUSSIAN, 2.0), _t(Y), s, 9, 77, _t(x_c), rho, _t(proj),
                                              _t(th), ex_begin=0, ex_end=128, pool_rows=pool_rows)
        rows_g = rows_g.cpu().numpy()
        assert fc == int(far.sum()) and st == ffc.FFC_OK and rows_g.size == s
        if prev is not None:
            assert list(rows_g[:prev.size]) == list(prev)      # keys do not depend on s
        prev = rows_g
        pool = oprop.candidate_pool(far, 9, 77, pool_rows)
        assert np.unique(rows_g).size == s and set(rows_g) <= set(pool)
        # keys of the oracle (FP64 network); the GPU's FP32 logits may only
        # swap rows whose keys are within the logits' rounding of the cut
        F = oprop.features(Y, pool, x_c, rho, kern, proj)
        o, _ = omlp.forward(omlp.half_weights(th), F)
        keys = oprop.es_keys(oprop.mixed_weights(o), 9, 77)
        pos = {int(r): i for i, r in enumerate(pool)}
        sel = np.array([pos[int(r)] for r in rows_g])
        cut = np.sort(keys)[::-1][s - 1]
        margin = 1e-3 * abs(cut)
        assert np.min(keys[sel]) >= cut - margin
        rest = np.setdiff1d(np.arange(pool.size), sel)
        assert np.max(keys[rest]) <= cut + margin
        rows_o = oprop.propose_from_mask(far, Y, s, 9, 77, x_c, rho, kern, proj, th, pool_rows)
        assert len(set(rows_o) ^ set(rows_g)) <= max(2, s // 50)
    # a far field of at most s rows is taken whole
    small_Y = Y[:128 + 30]
    rows_g, fc, st = ffc.ffc_propose_rows(ffc.Kernel(GAUSSIAN, 2.0), _t(small_Y), 64, 9, 77, _t(x_c), rho,
                                          _t(proj), _t(th), ex_begin=0, ex_end=128)
    far_s = np.flatnonzero(far_field_mask(small_Y, x_c, rho, 1.0, 0, 128))
    assert st == ffc.FFC_E_FARFIELD_TOO_SMALL and sorted(rows_g.cpu().numpy()) == list(far_s)


def _gram_error(n, s1):
    """Bound on the perturbation of K^T K from its FP64 sums and the Jacobi
    rotations: 10 n eps ||K||_2^2."""
    return 10.0 * n * 2.220446049250313e-16 * s1 * s1


def _lev_check(ffc, K, eps, r_fixed=0):
    Kcm = _t(K.T.copy())
    lev, sig, r, st = ffc.ffc_leverage(Kcm, eps, r_fixed)
    lev, sig = lev.cpu().numpy(), sig.cpu().numpy()
    so = singular_values(K)
    ro = r_fixed if r_fixed > 0 else int(np.sum(so >= eps * so[0]))
    assert st == ffc.FFC_OK and r == ro
    s1 = so[0]
    E = _gram_error(K.shape[1], s1)
    # Weyl: |lambda_gpu - sigma^2| <= E, so |sigma_gpu - sigma| <= E / max(sigma, sqrt(E))
    tol_sig = E / np.maximum(so, np.sqrt(E)) + 1e-15 * s1
    assert np.all(np.abs(sig[:so.size] - so) <= tol_sig)
    U, _, _ = np.linalg.svd(K, full_matrices=False)
    lo = np.sum(U[:, :r] ** 2, axis=1)
    # Davis-Kahan: the rank-r subspace moves by at most E / gap
    gap = so[r - 1] ** 2 - (so[r] ** 2 if r < so.size else 0.0)
    bound = 2.0 * E / gap + 1e-12
    assert np.max(np.abs(lev - lo)) <= bound
    assert abs(lev.sum() - r) <= 1e-6 * r + r * bound
    return r, bound


def test_leverage_matches_oracle(ffc):
    K = workloads.random_matrix(2000, 150, seed=3, decay=0.8)
    r, bound = _lev_check(ffc, K, 1e-4)
    assert r == 42 and bound < 1e-3
    _lev_check(ffc, K, 1e-6)
    _lev_check(ffc, K, 0.0, r_fixed=10)
    # ragged and degenerate shapes: odd n (unpaired index), m below one tile, one column
    _lev_check(ffc, workloads.random_matrix(37, 9, seed=4), 1e-8)
    _lev_check(ffc, workloads.random_matrix(500, 257, seed=5, decay=0.95), 1e-3)
    _lev_check(ffc, workloads.random_matrix(300, 1, seed=6), 1e-8)


def test_leverage_of_a_kernel_block(ffc):
    Y, x_c, rho = _node(seed=4, N=4096, n=256)
    far = np.flatnonzero(far_field_mask(Y, x_c, rho, 1.0, 0, 256))
    from oracle.kernels import kernel_block
    K, _ = kernel_block(Kernel(GAUSSIAN, h=2.0), Y[far], Y[:256])
    Kcm = _t(K.T.copy())
    lev, sig, r, st = ffc.ffc_leverage(Kcm, 1e-6)
    to, ro = oprop.leverage_targets(K, 1e-6)
    so = singular_values(K)
    near = np.abs(so / so[0] - 1e-6) < 1e-3 * 1e-6
    if not np.any(near):
        assert r == ro
    lev = lev.cpu().numpy()
    assert np.all(lev >= -1e-9) and np.all(lev <= 1 + 1e-9) and abs(lev.sum() - r) < 1e-6 * r
    gap = so[r - 1] ** 2 - (so[r] ** 2 if r < so.size else 0.0)
    assert np.max(np.abs(lev / r - to)) <= 2.0 * _gram_error(256, so[0]) / gap / r + 1e-10


def test_training_steps_match_oracle(ffc):
    g = np.random.default_rng(12)
    sizes = [300, 200, 100]
    off = np.concatenate([[0], np.cumsum(sizes)])
    R = int(off[-1])
    F = (1.2 * g.standard_normal((R, 12))).astype(np.float32)
    t = g.random(R) ** 4
    th0 = _params(13)
    lr = 3e-3
    # GPU
    tg = _t(th0); mg = torch.zeros_like(tg); vg = torch.zeros_like(tg)
    losses_g = []
    for step in range(1, 6):
        loss, grad = ffc.ffc_mlp_loss_grad(tg, _t(F), _t(t), _t(off, torch.int64))
        ffc.ffc_adam_step(tg, grad, mg, vg, step, lr)
        losses_g.append(loss)
    # oracle with the same FP32 storage of parameters and moments
    th = th0.copy(); m = np.zeros_like(th); v = np.zeros_like(th)
    losses_o = []
    for step in range(1, 6):
        loss, grad = omlp.loss_and_grad(th, F.astype(np.float64), t, off, half=True)
        th64, m64, v64 = omlp.adam_step(th, grad.astype(np.float32), m, v, step, lr)
        th, m, v = th64.astype(np.float32), m64.astype(np.float32), v64.astype(np.float32)
        losses_o.append(loss)
    np.testing.assert_allclose(losses_g, losses_o, rtol=1e-4)
    assert losses_g[-1] < losses_g[0]
    diff = np.linalg.norm(tg.cpu().numpy() - th) / np.linalg.norm(th0)
    assert diff < 2e-3


def _tree_nodes(ffc, X, leaf, levels, count, seed):
    Xd = _t(X)
    tree = ffc.ffc_build_tree(Xd, leaf)
    Xp = Xd[tree.perm].contiguous()
    lv = np.floor(np.log2(np.arange(tree.n_nodes) + 1)).astype(int)
    cand = np.flatnonzero(np.isin(lv, levels))
    pick = np.random.default_rng(seed).choice(cand, size=min(count, cand.size), replace=False)
    return Xp, tree, sorted(int(i) for i in pick)


def test_learned_proposal_gains_over_uniform(ffc):
    """Train on the d=128 (Laplace) and d=1000 (Gaussian) generators, compare
    full-block ID errors with uniform sampling at equal s on held-out seeds."""
    from paper_1409_2802_gb300 import learned

    def median_distance(X, k=400):
        S = X[:k].astype(np.float64)
        d2 = np.sum((S[:, None] - S[None]) ** 2, axis=2)
        return float(np.median(np.sqrt(d2[np.triu_indices(k, 1)])))

    def sources(seed):
        X3 = workloads.decaying_mixture(16384, 128, 16, seed=seed)
        X4 = workloads.low_intrinsic(16384, 10, 1000, seed=seed)
        k3 = ffc.Kernel(ffc.LAPLACE)
        k4 = ffc.Kernel(ffc.GAUSSIAN, h=median_distance(X4))
        out = []
        for X, leaf, k, lv in ((X3, 256, k3, [5, 6]), (X4, 512, k4, [5])):
            Xp, tree, nodes = _tree_nodes(ffc, X, leaf, lv, 12, seed)
            out.append((Xp, tree, nodes, k, _t(workloads.projections(X.shape[1], seed=7))))
        return out

    ts = learned.build_training_set(sources(0), eps=1e-6, batch_nodes=4, seed=0)
    th0 = workloads.mlp_init(1)
    loss0 = learned.mean_loss(ts, _t(th0))
    params, losses = learned.train(ts, th0, epochs=40, lr=2e-3, seed=0)
    loss1 = learned.mean_loss(ts, params)
    assert loss1 < loss0

    s = 128
    errs = {"uniform": [], "learned": []}
    for Xp, tree, nodes, k, proj in sources(1000):
        for node in nodes[:8]:
            b = int(tree.begin[node].item()); n = int(tree.count[node].item())
            x_c = tree.centroid[node].contiguous(); rho = float(tree.radius[node].item())
            far = ffc.ffc_far_field(Xp, x_c, rho, 1.0, b, b + n)
            if far.numel() < 8 * s:
                continue
            for mode in errs:
                if mode == "uniform":
                    rows, _, _ = ffc.ffc_sample_rows(Xp, s, 5, node, x_c, rho, 1.0, b, b + n)
                else:
                    rows, _, _ = ffc.ffc_propose_rows(k, Xp, s, 5, node, x_c, rho, proj, params, 1.0, b, b + n,
                                                      pool_rows=0)
                Kc, _ = ffc.ffc_eval_block(k, Xp, rows, Xp[b:b + n])
                Kst = Kc.t().contiguous()
                skel, T, r, _, _ = ffc.ffc_id(Kst, s // 2, 1e-6)
                e = ffc.ffc_id_error(k, Xp, Xp[b:b + n], skel, T, r, rows=far)
                errs[mode].append(max(e, 1e-16))
    lu, ll = np.log10(errs["uniform"]), np.log10(errs["learned"])
    print(f"held-out nodes {lu.size}: median log10 full-block error uniform {np.median(lu):.2f}, "
          f"learned {np.median(ll):.2f}; training loss {loss0:.3f} -> {loss1:.3f}")
    assert lu.size >= 8
    assert np.median(ll) < np.median(lu) - 0.5
