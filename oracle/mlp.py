"""FP64 CPU oracle of the triage network -- TEST INFRASTRUCTURE ONLY.

Only the tests, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline
leg may import this module; the product library never does.

The network is a three-layer perceptron (the paper has no learned part; this
is the surrogate that triages a ligand stream):

    x_hat = (x - mu) / sigma                       [nin]
    h1    = relu(W1 x_hat + b1)                    [256]
    h2    = relu(W2 h1 + b2)                       [256]
    y     = w3 . h2 + b3                           (normalised prediction)
    loss  = (1/B) sum_b (y_b - (t_b - mu_y) / sigma_y)^2

written as plain numpy matrix products in float64.  Parameters are packed in
the order W1 [256][nin], b1 [256], W2 [256][256], b2 [256], w3 [256], b3 [1].

With ``bf16=True`` the oracle rounds, to bfloat16 (round to nearest, ties to
even), exactly the quantities a BF16-weight / FP32-accumulate implementation
stores in BF16: x_hat, W1, W2, w3, h1, and the back-propagated dh2 and dh1
where they enter a product.  The bias gradients and dW3 use the unrounded
values.  ``bf16=False`` is the plain FP64 network (used for the
finite-difference pins).

Optimiser: Adam (Kingma & Ba 2015): m <- b1 m + (1-b1) g, v <- b2 v + (1-b2) g^2,
theta <- theta - lr * (m / (1-b1^t)) / (sqrt(v / (1-b2^t)) + eps).
"""
from __future__ import annotations

import numpy as np

HIDDEN = 256


def bf16(a):
    """Round to the nearest bfloat16 (ties to even), returned as float64.
    The value is first rounded to float32 (as a float32 computation holds
    it), then its low 16 bits are rounded away."""
    f = np.asarray(a, dtype=np.float64).astype(np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> np.uint64(16)) & np.uint64(1)
    r = ((u + np.uint64(0x7FFF) + lsb) & np.uint64(0xFFFF0000)).astype(np.uint32)
    return r.view(np.float32).astype(np.float64)


def nparams(nin: int) -> int:
    return HIDDEN * nin + HIDDEN + HIDDEN * HIDDEN + HIDDEN + HIDDEN + 1


def unpack(theta, nin: int):
    theta = np.asarray(theta, np.float64)
    o = 0
    W1 = theta[o:o + HIDDEN * nin].reshape(HIDDEN, nin); o += HIDDEN * nin
    b1 = theta[o:o + HIDDEN]; o += HIDDEN
    W2 = theta[o:o + HIDDEN * HIDDEN].reshape(HIDDEN, HIDDEN); o += HIDDEN * HIDDEN
    b2 = theta[o:o + HIDDEN]; o += HIDDEN
    w3 = theta[o:o + HIDDEN]; o += HIDDEN
    b3 = theta[o]
    return W1, b1, W2, b2, w3, b3


def pack(W1, b1, W2, b2, w3, b3):
    return np.concatenate([np.ravel(W1), b1, np.ravel(W2), b2, w3, [b3]]).astype(np.float64)


def forward(theta, x, nin, mu, sigma, bf16_storage=True):
    """Normalised predictions y [B] and the intermediate values."""
    W1, b1, W2, b2, w3, b3 = unpack(theta, nin)
    r = bf16 if bf16_storage else (lambda a: np.asarray(a, np.float64))
    xh = r((np.asarray(x, np.float64) - mu) / sigma)
    W1r, W2r, w3r = r(W1), r(W2), r(w3)
    z1 = xh @ W1r.T + b1
    h1 = r(np.maximum(z1, 0.0))
    z2 = h1 @ W2r.T + b2
    h2 = np.maximum(z2, 0.0)
    y = h2 @ w3r + b3
    return y, dict(xh=xh, h1=h1, h2=h2, W1r=W1r, W2r=W2r, w3r=w3r)


def loss_and_grad(theta, x, t, nin, mu, sigma, mu_y, sigma_y, bf16_storage=True):
    """Batch loss and its gradient with respect to the packed parameters."""
    r = bf16 if bf16_storage else (lambda a: np.asarray(a, np.float64))
    y, c = forward(theta, x, nin, mu, sigma, bf16_storage)
    B = len(y)
    th = (np.asarray(t, np.float64) - mu_y) / sigma_y
    res = y - th
    loss = float(np.sum(res * res) / B)
    dy = 2.0 * res / B                                   # dL/dy
    g_b3 = dy.sum()
    g_w3 = c["h2"].T @ dy                                # sum_b dy_b h2_b
    dh2 = np.outer(dy, c["w3r"]) * (c["h2"] > 0)         # dL/dz2
    g_b2 = dh2.sum(axis=0)
    dh2r = r(dh2)
    g_W2 = dh2r.T @ c["h1"]                              # [out][in]
    dh1 = (dh2r @ c["W2r"]) * (c["h1"] > 0)              # dL/dz1
    g_b1 = dh1.sum(axis=0)
    dh1r = r(dh1)
    g_W1 = dh1r.T @ c["xh"]
    return loss, pack(g_W1, g_b1, g_W2, g_b2, g_w3, g_b3)


def adam(theta, m, v, g, step, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update (step counts from 1); returns new theta, m, v."""
    m = beta1 * m + (1.0 - beta1) * g
    v = beta2 * v + (1.0 - beta2) * g * g
    mh = m / (1.0 - beta1 ** step)
    vh = v / (1.0 - beta2 ** step)
    return theta - lr * mh / (np.sqrt(vh) + eps), m, v
