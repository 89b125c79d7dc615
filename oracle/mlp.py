"""CPU oracle of the warm-start network: a plain NumPy FP64 multilayer perceptron.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Network (3 weight layers): H1 = tanh(X W1 + b1), H2 = tanh(H1 W2 + b2), Y = H2 W3 + b3.
Loss: L = sum((Y - T)^2) / (N n_out) (mean squared error over samples and outputs).
Gradients by the chain rule written out layer by layer.  Parameters are one flat vector in the
order W1 (n_in x n_h, row-major), b1, W2 (n_h x n_h), b2, W3 (n_h x n_out), b3 - the layout of the
GPU network's parameter buffer.
"""
from __future__ import annotations

import numpy as np


def shapes(n_in: int, n_h: int, n_out: int):
    return [(n_in, n_h), (n_h,), (n_h, n_h), (n_h,), (n_h, n_out), (n_out,)]


def unflatten(theta, n_in, n_h, n_out):
    out, o = [], 0
    for s in shapes(n_in, n_h, n_out):
        k = int(np.prod(s))
        out.append(np.asarray(theta[o:o + k], np.float64).reshape(s))
        o += k
    return out


def flatten(parts):
    return np.concatenate([np.asarray(p, np.float64).ravel() for p in parts])


def forward(theta, X, n_in, n_h, n_out):
    W1, b1, W2, b2, W3, b3 = unflatten(theta, n_in, n_h, n_out)
    H1 = np.tanh(X @ W1 + b1)
    H2 = np.tanh(H1 @ W2 + b2)
    return H2 @ W3 + b3, (X, H1, H2)


def loss_and_grad(theta, X, T, n_in, n_h, n_out):
    W1, b1, W2, b2, W3, b3 = unflatten(theta, n_in, n_h, n_out)
    Y, (X_, H1, H2) = forward(theta, X, n_in, n_h, n_out)
    N = X.shape[0]
    R = Y - T
    L = float(np.sum(R * R) / (N * n_out))
    dY = 2.0 * R / (N * n_out)
    dW3 = H2.T @ dY
    db3 = dY.sum(axis=0)
    dZ2 = (dY @ W3.T) * (1.0 - H2 * H2)
    dW2 = H1.T @ dZ2
    db2 = dZ2.sum(axis=0)
    dZ1 = (dZ2 @ W2.T) * (1.0 - H1 * H1)
    dW1 = X_.T @ dZ1
    db1 = dZ1.sum(axis=0)
    return L, flatten([dW1, db1, dW2, db2, dW3, db3])
