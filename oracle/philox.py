"""Philox4x64-10 counter-based random numbers (oracle side).

Test infrastructure (see ``oracle/__init__``).

Definition (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy as
1, 2, 3", SC'11): a 256-bit counter X = (x0, x1, x2, x3) and a 128-bit key
(k0, k1). One round multiplies x0 and x2 by the constants M0 and M1 into
128-bit products and recombines the halves:

    (hi0, lo0) = M0 * x0,  (hi1, lo1) = M1 * x2
    X <- (hi1 ^ x1 ^ k0,  lo1,  hi0 ^ x3 ^ k1,  lo0)

and between rounds the key is bumped by the Weyl constants (W0, W1). Ten
rounds give the four 64-bit output words.

Stream layout used by the method: draw t of stream (seed, stream_id, domain)
is word (t mod 4) of Philox(counter = (t // 4, stream_id, domain, 0),
key = (seed, 0)).
"""
from __future__ import annotations

import numpy as np

M0 = 0xD2E7470EE14C6C93
M1 = 0xCA5A826395121157
W0 = 0x9E3779B97F4A7C15
W1 = 0xBB67AE8584CAA73B
_MASK = (1 << 64) - 1

# counter domains of the draws the method makes
DOMAIN_UNIFORM_ROWS = 0      # uniform far-field row sampling
DOMAIN_WEIGHTED_POOL = 1     # candidate pool of the learned proposal
DOMAIN_WEIGHTED_KEYS = 2     # Efraimidis-Spirakis keys of the weighted sampler
DOMAIN_PAPER_SAMPLERS = 3    # keys of the paper's distance and leverage samplers (oracle/samplers.py)


def philox4x64_10(counter, key):
    """One Philox4x64-10 block with Python integers (scalar reference form)."""
    x = [int(c) & _MASK for c in counter]
    k0, k1 = int(key[0]) & _MASK, int(key[1]) & _MASK
    for _ in range(10):
        p0 = M0 * x[0]
        p1 = M1 * x[2]
        x = [((p1 >> 64) ^ x[1] ^ k0) & _MASK, p1 & _MASK,
             ((p0 >> 64) ^ x[3] ^ k1) & _MASK, p0 & _MASK]
        k0 = (k0 + W0) & _MASK
        k1 = (k1 + W1) & _MASK
    return x


def _mulhilo(a: np.ndarray, b: int):
    """128-bit product of uint64 array a and constant b, as (hi, lo) uint64."""
    a = a.astype(np.uint64)
    m32 = np.uint64(0xFFFFFFFF)
    s32 = np.uint64(32)
    bl, bh = np.uint64(b & 0xFFFFFFFF), np.uint64(b >> 32)
    al, ah = a & m32, a >> s32
    ll = al * bl
    lh = al * bh
    hl = ah * bl
    hh = ah * bh
    mid = (ll >> s32) + (lh & m32) + (hl & m32)
    hi = hh + (lh >> s32) + (hl >> s32) + (mid >> s32)
    lo = a * np.uint64(b)          # wraps modulo 2**64
    return hi, lo


def philox4x64_10_np(c0, c1, c2, c3, k0: int, k1: int):
    """Vectorised Philox4x64-10 over arrays of counters; returns 4 uint64 arrays."""
    with np.errstate(over="ignore"):
        x0 = np.asarray(c0, dtype=np.uint64).copy()
        x1 = np.broadcast_to(np.asarray(c1, dtype=np.uint64), x0.shape).copy()
        x2 = np.broadcast_to(np.asarray(c2, dtype=np.uint64), x0.shape).copy()
        x3 = np.broadcast_to(np.asarray(c3, dtype=np.uint64), x0.shape).copy()
        ka, kb = int(k0) & _MASK, int(k1) & _MASK
        for _ in range(10):
            hi0, lo0 = _mulhilo(x0, M0)
            hi1, lo1 = _mulhilo(x2, M1)
            x0, x1, x2, x3 = hi1 ^ x1 ^ np.uint64(ka), lo1, hi0 ^ x3 ^ np.uint64(kb), lo0
            ka = (ka + W0) & _MASK
            kb = (kb + W1) & _MASK
    return x0, x1, x2, x3


def draws(seed: int, stream_id: int, domain: int, t0: int, count: int) -> np.ndarray:
    """Draws t0 .. t0+count-1 of stream (seed, stream_id, domain) as uint64."""
    if count <= 0:
        return np.zeros(0, dtype=np.uint64)
    b0 = t0 // 4
    b1 = (t0 + count - 1) // 4
    blocks = np.arange(b0, b1 + 1, dtype=np.uint64)
    w = philox4x64_10_np(blocks, stream_id, domain, 0, seed, 0)
    flat = np.stack(w, axis=1).reshape(-1)          # word-major within a block
    off = t0 - 4 * b0
    return flat[off:off + count]


def mulhi_index(w: np.ndarray, M: int) -> np.ndarray:
    """floor(w * M / 2**64): maps a uniform 64-bit word to an index in [0, M)."""
    return np.array([(int(x) * int(M)) >> 64 for x in np.atleast_1d(w)], dtype=np.int64)


def to_unit_double(w: np.ndarray) -> np.ndarray:
    """(top 53 bits of w + 0.5) * 2**-53: a uniform double in (0, 1)."""
    top = (np.asarray(w, dtype=np.uint64) >> np.uint64(11)).astype(np.float64)
    return (top + 0.5) * (2.0 ** -53)
