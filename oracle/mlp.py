"""The proposer's multilayer perceptron in plain numpy FP64: forward pass,
backward pass (gradients of the mean squared error) and one Adam step.

Architecture: x (64) -> ReLU(W1 x + b1) (256) -> ReLU(W2 h1 + b2) (256) ->
ReLU(W3 h2 + b3) (256) -> W4 h3 + b4 (9).  Layer l maps d_in to d_out with
W_l of shape (d_out, d_in).  Loss L = (1/(B d)) sum_{batch, outputs}
(y - t)^2 over a batch of B samples with d = 9 outputs.  Adam (Kingma & Ba,
ICLR 2015): m <- b1 m + (1 - b1) g, v <- b2 v + (1 - b2) g^2,
w <- w - lr (m / (1 - b1^s)) / (sqrt(v / (1 - b2^s)) + eps) at step s.

Test infrastructure only (see quadrature.py).
"""
from __future__ import annotations

import numpy as np

LAYERS = [(64, 256), (256, 256), (256, 256), (256, 9)]


def init_params(seed=0, layers=LAYERS):
    """He-normal weights, zero biases (the same generator feeds both sides)."""
    rng = np.random.default_rng(seed)
    ps = []
    for din, dout in layers:
        ps.append(rng.standard_normal((dout, din)) * np.sqrt(2.0 / din))
        ps.append(np.zeros(dout))
    return ps


def forward(ps, X):
    """Outputs (B x 9) and the activations each layer saw (for backward)."""
    acts = [X]
    h = X
    nl = len(ps) // 2
    for l in range(nl):
        W, b = ps[2 * l], ps[2 * l + 1]
        z = h @ W.T + b[None, :]
        h = np.maximum(z, 0.0) if l < nl - 1 else z
        acts.append(h)
    return h, acts


def loss(ps, X, T):
    Y, _ = forward(ps, X)
    return float(np.mean((Y - T) ** 2))


def backward(ps, X, T):
    """Gradients of loss(ps, X, T) with respect to every parameter."""
    Y, acts = forward(ps, X)
    B, d = Y.shape
    delta = 2.0 * (Y - T) / (B * d)
    nl = len(ps) // 2
    grads = [None] * len(ps)
    for l in range(nl - 1, -1, -1):
        h_in = acts[l]
        grads[2 * l] = delta.T @ h_in
        grads[2 * l + 1] = delta.sum(axis=0)
        if l > 0:
            delta = (delta @ ps[2 * l]) * (acts[l] > 0.0)
    return grads


def adam_step(ps, grads, m, v, step, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update in place (step counts from 1)."""
    for i in range(len(ps)):
        m[i] = b1 * m[i] + (1.0 - b1) * grads[i]
        v[i] = b2 * v[i] + (1.0 - b2) * grads[i] ** 2
        mh = m[i] / (1.0 - b1 ** step)
        vh = v[i] / (1.0 - b2 ** step)
        ps[i] = ps[i] - lr * mh / (np.sqrt(vh) + eps)
    return ps
