"""The error bound behind the weighted draw's FP32 pre-selection, checked in IEEE FP32 on the host.

The draw ranks a large pool by FP32 keys k~ = L~ / w~' and computes FP64 keys only for the rows whose
k~ can be among the selection. It relies on |k~ - k| <= 9.5 u k (u = 2^-24), below its margin
DELTA = 2^-18, where k = -ln(u_d) / w' is the FP64 key (Efraimidis & Spirakis' key of the weighted
draw, with the uniform u_d = fl(m + 1/2) 2^-53 of the top 53 bits m of the draw). This test restates
the FP32 steps with numpy's float32 arithmetic (correctly rounded conversions, division and fma, and a
log within one ulp, the bound the derivation assumes):
* u_d rebuilt from the integer draw: (2m + 1) 2^-54 when m < 2^52; otherwise m + 1/2 rounds to the even
  neighbour m_e and 1 - u_d = (2^53 - m_e) 2^-53, both exact as integers;
* L~ = -log(u~) below 1/2, -log1p(-v~) above it: within 1.443 u + 2 u of -ln(u_d);
* w~' = 0.9 w~ / m~ + 0.1 in FP32: within 5 u of w';
* the key: within 9.5 u.
The GPU tests check the kernel itself (the draws equal the oracle's, the clustered-key fallback).
"""
import numpy as np

U = 2.0 ** -24


def _l_tilde(m):
    m = np.asarray(m, dtype=np.uint64)
    lo = m < np.uint64(1 << 52)
    L = np.empty(m.shape, np.float32)
    L[lo] = -np.log((2 * m[lo] + np.uint64(1)).astype(np.float64).astype(np.float32) * np.float32(2.0 ** -54))
    me = m[~lo] + (m[~lo] & np.uint64(1))
    v = (np.uint64(1 << 53) - me).astype(np.float64).astype(np.float32) * np.float32(2.0 ** -53)
    L[~lo] = -np.log1p(-v)
    return L


def _u_d(m):
    return (np.asarray(m, dtype=np.uint64).astype(np.float64) + 0.5) * 2.0 ** -53


def test_uniform_rebuild_and_log_within_the_bound():
    g = np.random.default_rng(3)
    m = g.integers(0, 1 << 53, size=400_000, dtype=np.uint64)
    edges = np.array([0, 1, 2, (1 << 52) - 2, (1 << 52) - 1, 1 << 52, (1 << 52) + 1, (1 << 53) - 3,
                      (1 << 53) - 2, (1 << 53) - 1], dtype=np.uint64)
    m = np.concatenate([m, edges])
    L = -np.log(_u_d(m))
    Lt = _l_tilde(m).astype(np.float64)
    zero = L == 0.0
    # u_d = 1 exactly (m + 1/2 rounds up to 2^53) gives the key 0 on both sides
    assert np.array_equal(zero, Lt == 0.0) and zero[-1]
    rel = np.abs(Lt[~zero] - L[~zero]) / L[~zero]
    assert rel.max() <= 3.443 * U, rel.max() / U


def test_key_within_the_preselection_margin():
    g = np.random.default_rng(4)
    n = 400_000
    m = g.integers(0, 1 << 53, size=n, dtype=np.uint64)
    w = np.exp(-g.exponential(6.0, size=n))        # weights exp(o - max o) in (0, 1]
    w[:3] = [1.0, 1e-45, 0.0]                        # the maximum, below the FP32 range, zero
    mean = w.mean()
    wp = 0.9 * w / mean + 0.1
    k = -np.log(_u_d(m)) / wp
    ratio = w.astype(np.float32) / np.float32(mean)
    wpt = (np.float32(0.9) * ratio.astype(np.float64) + np.float64(np.float32(0.1))).astype(np.float32)  # fmaf
    kt = (_l_tilde(m) / wpt).astype(np.float64)
    pos = k > 0
    rel = np.abs(kt[pos] - k[pos]) / k[pos]
    assert rel.max() <= 9.5 * U, rel.max() / U
    assert 9.5 * U < 2.0 ** -18
    assert np.all(kt[~pos] == 0.0)
