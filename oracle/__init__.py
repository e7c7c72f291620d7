"""Plain FP64 CPU oracle for sampled-row far-field compression (March & Biros).

TEST INFRASTRUCTURE, NOT PART OF THE PRODUCT. Only ``tests/``,
``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline / reference leg may
import it. It shares no code with the CUDA path (``paper_1409_2802_gb300``) and
never imports it; the product path never imports this package.

Each function follows one step of the paper's method, written for a reader who
checks it against the paper by eye: no blocking, no fusion, no reordering.

* ``philox``    Philox4x64-10 counter-based generator (Salmon et al., SC'11),
                the source of every random number the method draws.
* ``sampling``  far field T = {y : ||y - x_c|| >= xi*rho} (§4.1) and uniform
                row sampling without replacement (§2.2, §4.1.3).
* ``kernels``   Gaussian (§4.2), Laplace (§4.3) and polynomial (§4.4) kernels.
* ``cpqr``      Businger-Golub column-pivoted Householder QR (§2.1.3, App. A.1).
* ``interp``    the interpolative decomposition from the pivoted QR
                (Def. "Interpolative Decomposition", §2.1.3; App. A.1) and its
                full-block reconstruction error (§4.1.3 step 4).
* ``spectral``  truncated-SVD error and epsilon-rank (§2.1.3, §4.1.3 step 1),
                statistical leverage scores and coherence (§3).
* ``tree``      PCA median-split binary tree and per-node far-field geometry.
* ``compress``  per-node sampled ID over all tree levels >= 2.
* ``mlp``       FP64 forward/backward/Adam of the learned sampling proposal.
* ``proposal``  its features, weighted sampling without replacement and the
                leverage-score training targets (§3, §4.1.3).
* ``apply``     the outgoing representation: skeleton charges q~ = P q and the
                far-field potential C q~ (§2.1.3).
* ``samplers``  the paper's other row samplers: distance, leverage and nearest
                neighbours (§4.1.3, §3).

Parity pins live in ``tests/test_oracle_*.py``. Parts without an independent
pin are marked "parity unpinned" in their module docstring.
"""
