"""FP64 forward pass, backward pass and Adam step of the learned sampling proposal.

Test infrastructure (see ``oracle/__init__``).

The proposal network is not in the paper. It stands in for the leverage-score
importance distribution of §3 (Def. "Statistical Leverage"; §4.1.3 "Leverage
sampling"), which the paper shows to be the best row distribution but which
needs the SVD of the full block. The network maps 12 cheap per-row features to
a logit o_i, and the proposal is softmax(o) over a node's far-field rows.

Network: x (12) -> z1 = W1 x + b1 -> h1 = GELU(z1) (128)
                -> z2 = W2 h1 + b2 -> h2 = GELU(z2) (128) -> o = w3 . h2 + b3.
GELU(z) = z Phi(z) = z (1 + erf(z / sqrt 2)) / 2 (Hendrycks & Gimpel, erf form).

Loss of a batch of B nodes (rows of node b in [off[b], off[b+1])), targets
t >= 0 normalised per node to the distribution q_i = t_i / sum_{j in b} t_j
(for leverage scores, q = l / r):
    L = (1/B) sum_b  -sum_{i in b} q_i log softmax_b(o)_i,
the cross-entropy between the target distribution and the network's proposal.
A node whose targets sum to zero contributes nothing.

Adam: Kingma & Ba (ICLR 2015), Algorithm 1, with bias-corrected moments.

Precision reading: the network's weights are stored as an FP32 master copy
and used in the forward and backward passes rounded to FP16 (round to
nearest even); ``half_weights`` gives those FP16 values as exact float64
numbers, and everything after that is FP64 here: the activations are not
rounded, in inference or in training.
"""
from __future__ import annotations

import numpy as np
from scipy.special import erf

N_IN = 12
N_HID = 128
LAYOUT = {
    "W1": (0, (N_HID, N_IN)),
    "b1": (1536, (N_HID,)),
    "W2": (1664, (N_HID, N_HID)),
    "b2": (18048, (N_HID,)),
    "w3": (18176, (N_HID,)),
    "b3": (18304, (1,)),
}
N_PARAMS = 18305

_SQRT2 = np.sqrt(2.0)
_INV_SQRT_2PI = 1.0 / np.sqrt(2.0 * np.pi)


def unpack(theta) -> dict:
    """Views of the flat parameter vector as float64 arrays."""
    theta = np.asarray(theta, dtype=np.float64)
    out = {}
    for name, (off, shape) in LAYOUT.items():
        size = int(np.prod(shape))
        out[name] = theta[off:off + size].reshape(shape)
    return out


def pack(parts: dict) -> np.ndarray:
    theta = np.zeros(N_PARAMS, dtype=np.float64)
    for name, (off, shape) in LAYOUT.items():
        size = int(np.prod(shape))
        theta[off:off + size] = np.asarray(parts[name], dtype=np.float64).reshape(size)
    return theta


def half_weights(theta32) -> np.ndarray:
    """The FP16 values the network computes with, as float64."""
    return np.asarray(theta32, dtype=np.float32).astype(np.float16).astype(np.float64)


def gelu(z):
    return 0.5 * z * (1.0 + erf(z / _SQRT2))


def gelu_prime(z):
    """d/dz [z Phi(z)] = Phi(z) + z phi(z)."""
    return 0.5 * (1.0 + erf(z / _SQRT2)) + z * _INV_SQRT_2PI * np.exp(-0.5 * z * z)


def forward(theta, X):
    """Logits o (R,) of the R x 12 feature rows X, and the cache for backward."""
    p = unpack(theta)
    X = np.asarray(X, dtype=np.float64)
    z1 = X @ p["W1"].T + p["b1"]
    h1 = gelu(z1)
    z2 = h1 @ p["W2"].T + p["b2"]
    h2 = gelu(z2)
    o = h2 @ p["w3"] + p["b3"][0]
    return o, (X, z1, h1, z2, h2)


def backward(theta, cache, g_o):
    """Gradient of sum_i g_o[i] * o_i with respect to every parameter (flat vector)."""
    p = unpack(theta)
    X, z1, h1, z2, h2 = cache
    g_o = np.asarray(g_o, dtype=np.float64)
    g = {}
    g["w3"] = h2.T @ g_o
    g["b3"] = np.array([np.sum(g_o)])
    g_h2 = np.outer(g_o, p["w3"])
    g_z2 = g_h2 * gelu_prime(z2)
    g["W2"] = g_z2.T @ h1
    g["b2"] = np.sum(g_z2, axis=0)
    g_h1 = g_z2 @ p["W2"]
    g_z1 = g_h1 * gelu_prime(z1)
    g["W1"] = g_z1.T @ X
    g["b1"] = np.sum(g_z1, axis=0)
    return pack(g)


def softmax_cross_entropy(o, t, node_off):
    """Mean over nodes of -sum q_i log softmax(o)_i (q = t / sum t per node), and dL/do."""
    o = np.asarray(o, dtype=np.float64)
    t = np.asarray(t, dtype=np.float64)
    B = len(node_off) - 1
    loss = 0.0
    g_o = np.zeros_like(o)
    for b in range(B):
        a, e = int(node_off[b]), int(node_off[b + 1])
        if e <= a:
            continue
        ob = o[a:e]
        mx = np.max(ob)
        lse = mx + np.log(np.sum(np.exp(ob - mx)))
        pb = np.exp(ob - lse)
        tsum = np.sum(t[a:e])
        if tsum <= 0.0:
            continue
        qb = t[a:e] / tsum
        loss += -np.sum(qb * (ob - lse))
        g_o[a:e] = pb - qb
    return loss / B, g_o / B


def loss_and_grad(theta32, X, t, node_off, half: bool = True):
    """Loss and flat FP64 gradient of the proposal network on one batch of nodes.

    With ``half`` the weights are the FP16 values of the FP32 master copy
    (the precision the network is used in); without it theta is used as is.
    """
    theta = half_weights(theta32) if half else np.asarray(theta32, dtype=np.float64)
    o, cache = forward(theta, X)
    loss, g_o = softmax_cross_entropy(o, t, node_off)
    return loss, backward(theta, cache, g_o)


def adam_step(theta, grad, m, v, step: int, lr: float, beta1: float = 0.9,
              beta2: float = 0.999, eps: float = 1e-8):
    """One Adam update (step counts from 1). Returns new (theta, m, v)."""
    g = np.asarray(grad, dtype=np.float64)
    m = beta1 * np.asarray(m, dtype=np.float64) + (1.0 - beta1) * g
    v = beta2 * np.asarray(v, dtype=np.float64) + (1.0 - beta2) * g * g
    m_hat = m / (1.0 - beta1 ** step)
    v_hat = v / (1.0 - beta2 ** step)
    theta = np.asarray(theta, dtype=np.float64) - lr * m_hat / (np.sqrt(v_hat) + eps)
    return theta, m, v
