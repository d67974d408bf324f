"""Warm-start network (oracle, test infrastructure).

The paper has no learned component; this is the reference for the multiplier
warm start of the GPU library: a 3-layer perceptron x -> lambda0 with ReLU
hidden layers, BF16 operands and FP32 (here FP64) accumulation, trained with
mean squared error and Adam.

Conventions shared with the CUDA kernels (the same arithmetic, written
independently):
  * layer l: Z_l = bf16(A_{l-1}) bf16(W_l)^T + b_l, A_l = relu(Z_l) (no
    activation on the last layer); W_l is (out x in), row-major;
  * loss = mean over batch and outputs of (Y - T)^2; dY = 2 (Y - T) / (B n_out);
  * backward: dW_l = bf16(dZ_l)^T bf16(A_{l-1}), db_l = column sums of dZ_l,
    dA_{l-1} = bf16(dZ_l) bf16(W_l), dZ_{l-1} = dA_{l-1} * [Z_{l-1} > 0];
  * Adam with beta1 = 0.9, beta2 = 0.999, eps = 1e-8, bias correction.
Parity: pinned by central finite differences of the loss in FP64 with the
roundings disabled (``test_oracle_mlp.py``).
"""
from __future__ import annotations

import numpy as np


def bf16(x: np.ndarray) -> np.ndarray:
    """Round to the nearest bfloat16 (ties to even), returned as float64."""
    a = np.asarray(x, np.float32)
    u = a.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    u = ((u + 0x7FFF + lsb) >> 16) << 16
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def init_params(n_in, n_hidden, n_out, seed):
    """He-style uniform initialisation from a seeded generator (same draws as
    the library, which receives these values through its parameter setter)."""
    rng = np.random.default_rng(seed)
    shapes = [(n_hidden, n_in), (n_hidden, n_hidden), (n_out, n_hidden)]
    params = []
    for (o, i) in shapes:
        lim = np.sqrt(6.0 / i)
        params.append(rng.uniform(-lim, lim, size=(o, i)))
        params.append(np.zeros(o))
    return params


def forward(params, X, round_bf16=True):
    r = bf16 if round_bf16 else (lambda a: a)
    W1, b1, W2, b2, W3, b3 = params
    Z1 = r(X) @ r(W1).T + b1
    A1 = np.maximum(Z1, 0)
    Z2 = r(A1) @ r(W2).T + b2
    A2 = np.maximum(Z2, 0)
    Y = r(A2) @ r(W3).T + b3
    return Y, (X, Z1, A1, Z2, A2)


def loss_and_grads(params, X, T, round_bf16=True):
    r = bf16 if round_bf16 else (lambda a: a)
    W1, b1, W2, b2, W3, b3 = params
    Y, (X, Z1, A1, Z2, A2) = forward(params, X, round_bf16)
    B, n_out = Y.shape
    loss = np.mean((Y - T) ** 2)
    dY = 2.0 * (Y - T) / (B * n_out)
    dW3 = r(dY).T @ r(A2)
    db3 = dY.sum(0)
    dA2 = r(dY) @ r(W3)
    dZ2 = dA2 * (Z2 > 0)
    dW2 = r(dZ2).T @ r(A1)
    db2 = dZ2.sum(0)
    dA1 = r(dZ2) @ r(W2)
    dZ1 = dA1 * (Z1 > 0)
    dW1 = r(dZ1).T @ r(X)
    db1 = dZ1.sum(0)
    return loss, [dW1, db1, dW2, db2, dW3, db3]


def adam_step(params, grads, state, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """In-place Adam update; state = (t, m list, v list)."""
    t, m, v = state
    t += 1
    for i, (p, g) in enumerate(zip(params, grads)):
        m[i] = beta1 * m[i] + (1 - beta1) * g
        v[i] = beta2 * v[i] + (1 - beta2) * g * g
        mh = m[i] / (1 - beta1 ** t)
        vh = v[i] / (1 - beta2 ** t)
        p -= lr * mh / (np.sqrt(vh) + eps)
    return (t, m, v)
