"""Pins for the oracle's Philox generator and uniform far-field sampler.

Philox is pinned to numpy's independent Philox4x64-10 implementation; the
sampler to the statistical properties that define uniform sampling without
replacement (§4.1.3 "Uniform sampling") and to a direct re-derivation of its
first accepted rows from the raw numpy stream.
"""
import numpy as np
import pytest

from oracle import philox
from oracle.sampling import ATTEMPT_FACTOR, far_field_mask, sample_uniform, sample_uniform_from_mask


def _numpy_block(key, ctr):
    """Philox4x64-10 block at counter ``ctr`` from numpy's own implementation.

    numpy adds one to the 256-bit counter before it generates a block, so it
    is started from ctr - 1 (with borrow across the four words).
    """
    v = sum(int(c) << (64 * i) for i, c in enumerate(ctr))
    v = (v - 1) % (1 << 256)
    prev = [(v >> (64 * i)) & (2**64 - 1) for i in range(4)]
    bg = np.random.Philox(key=np.array(key, dtype=np.uint64), counter=np.array(prev, dtype=np.uint64))
    return [int(x) for x in bg.random_raw(4)]


@pytest.mark.parametrize("key,ctr", [((0, 0), (0, 0, 0, 0)), ((5, 7), (1, 3, 0, 0)),
                                     ((2**64 - 1, 12345), (99, 2**63, 17, 3)),
                                     ((1, 2), (0, 4, 0, 0))])
def test_philox_scalar_matches_numpy(key, ctr):
    assert philox.philox4x64_10(ctr, key) == _numpy_block(key, ctr)


def test_philox_vectorised_matches_scalar():
    blocks = np.array([0, 1, 2, 1000, 2**40 + 3], dtype=np.uint64)
    out = philox.philox4x64_10_np(blocks, 9, 2, 0, 0xDEADBEEF, 0)
    for i, b in enumerate(blocks):
        ref = philox.philox4x64_10((int(b), 9, 2, 0), (0xDEADBEEF, 0))
        assert [int(o[i]) for o in out] == ref


def test_draw_layout_is_word_major():
    w = philox.draws(3, 11, 0, 0, 10)
    b0 = philox.philox4x64_10((0, 11, 0, 0), (3, 0))
    b1 = philox.philox4x64_10((1, 11, 0, 0), (3, 0))
    b2 = philox.philox4x64_10((2, 11, 0, 0), (3, 0))
    assert [int(x) for x in w] == (b0 + b1 + b2)[:10]
    assert [int(x) for x in philox.draws(3, 11, 0, 5, 3)] == (b0 + b1 + b2)[5:8]


def test_mulhi_index_exact():
    assert list(philox.mulhi_index(np.array([0, 2**63, 2**64 - 1], dtype=np.uint64), 1000)) == [0, 500, 999]
    assert list(philox.mulhi_index(np.array([2**62], dtype=np.uint64), 7)) == [1]


def _raw_candidates(seed, stream, count, M):
    """Candidate indices straight from numpy's Philox stream (independent path)."""
    out = []
    for b in range((count + 3) // 4):
        out += [(w * M) >> 64 for w in _numpy_block((seed, 0), (b, stream, 0, 0))]
    return out[:count]


def test_sampler_phase_a_rederived_from_numpy_stream():
    g = np.random.default_rng(1)
    Y = g.standard_normal((3000, 3))
    xc = np.zeros(3)
    far = far_field_mask(Y, xc, 1.0, 1.0, 100, 400)
    rows = sample_uniform_from_mask(far, 50, seed=12, stream_id=4)
    cand = _raw_candidates(12, 4, 2000, 3000)
    seen, expect = set(), []
    for j in cand:
        if far[j] and j not in seen:
            seen.add(j)
            expect.append(j)
        if len(expect) == 50:
            break
    assert list(rows) == expect


def test_sampler_distinct_far_prefix_consistent():
    # §4.1 setup: the sources are the n points nearest the centre
    g = np.random.default_rng(2)
    Y = g.standard_normal((5000, 4))
    Y = Y[np.argsort((Y * Y).sum(1))]
    xc = Y[:500].mean(axis=0)
    rho = float(np.sqrt(((Y[:500] - xc) ** 2).sum(1)).max())
    far = far_field_mask(Y, xc, rho, 1.0, 0, 500)
    assert not far[:500].any()
    r256, _ = sample_uniform(Y, 256, 7, 3, xc, rho, 1.0, 0, 500)
    r128, _ = sample_uniform(Y, 128, 7, 3, xc, rho, 1.0, 0, 500)
    assert len(set(r256.tolist())) == 256
    assert far[r256].all()
    assert np.array_equal(r256[:128], r128)


def test_sampler_small_far_field_takes_all():
    Y = np.arange(40, dtype=np.float64).reshape(-1, 1)
    rows, nfar = sample_uniform(Y, 64, 0, 0, x_c=np.zeros(1), radius=30.0)
    assert nfar == 10
    assert sorted(rows.tolist()) == list(range(30, 40))


def test_sampler_phase_b_fisher_yates():
    # 60 far candidates out of 20,000: acceptance 0.3%, so 64*s attempts run out
    M, s = 20000, 40
    far = np.zeros(M, dtype=bool)
    far[np.arange(0, M, M // 60)[:60]] = True
    rows = sample_uniform_from_mask(far, s, 5, 1)
    assert len(rows) == s and len(set(rows.tolist())) == s and far[rows].all()
    # phase B really ran: the phase-A stream alone does not yield s rows
    cand = philox.mulhi_index(philox.draws(5, 1, 0, 0, ATTEMPT_FACTOR * s), M)
    assert len({int(j) for j in cand if far[j]}) < s


def test_sampler_uniform_inclusion_chi2():
    M, s, trials = 200, 20, 4000
    far = np.ones(M, dtype=bool)
    far[:50] = False                          # 150 far candidates
    counts = np.zeros(M)
    for seed in range(trials):
        counts[sample_uniform_from_mask(far, s, seed, 0)] += 1
    assert counts[:50].sum() == 0
    obs = counts[50:]
    exp = trials * s / 150.0
    chi2 = float(((obs - exp) ** 2 / exp).sum())
    # 149 degrees of freedom (inclusions are weakly negatively correlated,
    # which only shrinks chi2); 99.99th percentile is about 227
    assert chi2 < 227.0, chi2
