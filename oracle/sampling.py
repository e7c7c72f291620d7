"""Far field and uniform row sampling without replacement (oracle side).

Test infrastructure (see ``oracle/__init__``).

Paper: the far field of a source set with centre x_c and radius rho is
T = {y : ||y - x_c|| >= xi * rho} (§4.1, experimental setup step 3); the method
forms the sampled block from s of the far-field targets chosen uniformly at
random without replacement (§2.2 "Our approach"; §4.1.3 "Uniform sampling").

Reading used here (the paper does not fix how the uniform subset is drawn):

* Candidates are the M rows of Y. A candidate is in the far field when it is
  outside the excluded index range [ex_begin, ex_end) (the node's own points
  in tree order) and sum_k (y_k - x_ck)^2 >= (xi*rho)^2. With no centre given,
  every non-excluded candidate is in the far field.
* Phase A (rejection): for t = 0, 1, ..., 64*s - 1 take draw w_t of the
  stream (seed, stream_id, DOMAIN_UNIFORM_ROWS), j = floor(w_t * M / 2^64);
  accept j if it is in the far field and not yet accepted; stop at s accepted.
  Rows are returned in acceptance order, so the first s' rows of a size-s
  sample are the size-s' sample (prefix consistency).
* Phase B (only if phase A ran out of attempts): T' = far-field candidates not
  yet accepted, ascending. If |T'| <= s - k take all of T'; otherwise a partial
  Fisher-Yates shuffle of T' with draws t = 64*s, 64*s + 1, ... picks the rest.

Each accepted row is uniform over the far field minus the rows already taken,
so the result is a uniform s-subset of T (or all of T when |T| <= s).
"""
from __future__ import annotations

import numpy as np

from .philox import DOMAIN_UNIFORM_ROWS, draws, mulhi_index

ATTEMPT_FACTOR = 64


def far_field_mask(Y, x_c=None, radius=0.0, xi=1.0, ex_begin=0, ex_end=0):
    """Boolean mask of the far-field candidates (§4.1 step 3)."""
    Y = np.asarray(Y, dtype=np.float64)
    M = Y.shape[0]
    mask = np.ones(M, dtype=bool)
    mask[ex_begin:ex_end] = False
    if x_c is not None:
        diff = Y - np.asarray(x_c, dtype=np.float64)[None, :]
        dist2 = np.sum(diff * diff, axis=1)
        thr = float(xi) * float(radius)
        mask &= dist2 >= thr * thr
    return mask


def sample_uniform(Y, s, seed, stream_id, x_c=None, radius=0.0, xi=1.0,
                   ex_begin=0, ex_end=0):
    """Uniform far-field row sample without replacement.

    Returns (rows int64[s_out], far_count) where s_out = min(s, |T|).
    """
    far = far_field_mask(Y, x_c, radius, xi, ex_begin, ex_end)
    return sample_uniform_from_mask(far, s, seed, stream_id), int(far.sum())


def sample_uniform_from_mask(far, s, seed, stream_id):
    M = far.shape[0]
    s = int(s)
    taken = np.zeros(M, dtype=bool)
    rows: list[int] = []
    attempts = ATTEMPT_FACTOR * s
    t = 0
    batch = 4096
    while len(rows) < s and t < attempts:
        cnt = min(batch, attempts - t)
        js = mulhi_index(draws(seed, stream_id, DOMAIN_UNIFORM_ROWS, t, cnt), M)
        for j in js:
            t += 1
            if far[j] and not taken[j]:
                taken[j] = True
                rows.append(int(j))
                if len(rows) == s:
                    break
    if len(rows) < s:
        rest = np.flatnonzero(far & ~taken)
        need = s - len(rows)
        if rest.size <= need:
            rows.extend(int(v) for v in rest)
        else:
            rest = rest.copy()
            w = draws(seed, stream_id, DOMAIN_UNIFORM_ROWS, attempts, need)
            for i in range(need):
                u = i + int(mulhi_index(w[i:i + 1], rest.size - i)[0])
                rest[i], rest[u] = rest[u], rest[i]
                rows.append(int(rest[i]))
    return np.asarray(rows, dtype=np.int64)
