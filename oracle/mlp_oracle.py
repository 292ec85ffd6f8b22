"""Plain FP64 CPU oracle of the learned interface warm start's network.

TEST INFRASTRUCTURE ONLY (see elm_oracle.py): only the tests import it.

y = W3^T g(W2^T g(W1^T x + b1) + b2) + b3 per sample (rows of X), g = GELU in its exact
form 0.5 z (1 + erf(z / sqrt 2)), loss L = sum (Y - T)^2 / (batch * d_out), and the
gradient of L with respect to every parameter by the chain rule written out layer by
layer.  Parameters are one flat vector in the order W1 [d_in][d_h], b1, W2 [d_h][d_h],
b2, W3 [d_h][d_out], b3 (row-major), as the library stores them.  The network, loss and
Adam rule are the standard ones; the paper has none of this (its interface solve is CG,
Section 4), so the oracle follows the definitions and is pinned by finite differences.
"""
from __future__ import annotations

import math

import numpy as np
from scipy.special import erf


def unpack(p, d_in, d_h, d_out):
    p = np.asarray(p, dtype=np.float64)
    o = 0
    out = []
    for shape in ((d_in, d_h), (d_h,), (d_h, d_h), (d_h,), (d_h, d_out), (d_out,)):
        n = int(np.prod(shape))
        out.append(p[o:o + n].reshape(shape))
        o += n
    assert o == p.size
    return out


def gelu(z):
    return 0.5 * z * (1.0 + erf(z / math.sqrt(2.0)))


def gelu_grad(z):
    return 0.5 * (1.0 + erf(z / math.sqrt(2.0))) + z * np.exp(-0.5 * z * z) / math.sqrt(2.0 * math.pi)


def forward(p, X, d_in, d_h, d_out):
    W1, b1, W2, b2, W3, b3 = unpack(p, d_in, d_h, d_out)
    z1 = X @ W1 + b1
    a1 = gelu(z1)
    z2 = a1 @ W2 + b2
    a2 = gelu(z2)
    return a2 @ W3 + b3, (z1, a1, z2, a2)


def loss_and_grad(p, X, T, d_in, d_h, d_out):
    W1, b1, W2, b2, W3, b3 = unpack(p, d_in, d_h, d_out)
    Y, (z1, a1, z2, a2) = forward(p, X, d_in, d_h, d_out)
    n = Y.size
    D = Y - T
    loss = float((D * D).sum() / n)
    dY = 2.0 * D / n
    gW3 = a2.T @ dY
    gb3 = dY.sum(0)
    d2 = (dY @ W3.T) * gelu_grad(z2)
    gW2 = a1.T @ d2
    gb2 = d2.sum(0)
    d1 = (d2 @ W2.T) * gelu_grad(z1)
    gW1 = X.T @ d1
    gb1 = d1.sum(0)
    g = np.concatenate([gW1.ravel(), gb1, gW2.ravel(), gb2, gW3.ravel(), gb3])
    return loss, g


def adam_step(p, g, m, v, step, lr, b1=0.9, b2=0.999, eps=1e-8):
    """Bias-corrected Adam (Kingma and Ba); returns (p, m, v) after one step."""
    m = b1 * m + (1.0 - b1) * g
    v = b2 * v + (1.0 - b2) * g * g
    lr_t = lr * math.sqrt(1.0 - b2 ** step) / (1.0 - b1 ** step)
    return p - lr_t * m / (np.sqrt(v) + eps), m, v
