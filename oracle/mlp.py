"""float64 reference of the nnz predictor network (test infrastructure only).

Network (this library's own definition; the paper has no predictor):
  h1 = relu(W1 x + b1)   W1: 32x8
  h2 = relu(W2 h1 + b2)  W2: 32x32
  y  = w3 . h2 + b3      w3: 32
Loss over a batch of N columns: L = (1/N) sum (y - t)^2 with t = log1p(nnz).
Adam (Kingma & Ba 2015) with bias correction updates every parameter.
Weight layout is row-major W[out][in], the same order the device kernels use.
"""
from __future__ import annotations

import numpy as np

SIZES = (8, 32, 32, 1)
NPARAM = 32 * 8 + 32 + 32 * 32 + 32 + 32 + 1


def unpack(theta: np.ndarray):
    o = 0
    W1 = theta[o:o + 256].reshape(32, 8); o += 256
    b1 = theta[o:o + 32]; o += 32
    W2 = theta[o:o + 1024].reshape(32, 32); o += 1024
    b2 = theta[o:o + 32]; o += 32
    w3 = theta[o:o + 32]; o += 32
    b3 = theta[o:o + 1]
    return W1, b1, W2, b2, w3, b3


def forward(theta, X):
    W1, b1, W2, b2, w3, b3 = unpack(np.asarray(theta, np.float64))
    X = np.asarray(X, np.float64)
    z1 = X @ W1.T + b1
    h1 = np.maximum(z1, 0.0)
    z2 = h1 @ W2.T + b2
    h2 = np.maximum(z2, 0.0)
    y = h2 @ w3 + b3[0]
    return y, (X, z1, h1, z2, h2)


def loss(theta, X, t):
    y, _ = forward(theta, X)
    return float(np.mean((y - np.asarray(t, np.float64)) ** 2))


def grad(theta, X, t):
    """Backpropagation of the mean squared error, by the chain rule layer by layer."""
    W1, b1, W2, b2, w3, b3 = unpack(np.asarray(theta, np.float64))
    y, (X, z1, h1, z2, h2) = forward(theta, X)
    N = X.shape[0]
    dy = 2.0 * (y - np.asarray(t, np.float64)) / N          # dL/dy
    g_w3 = h2.T @ dy
    g_b3 = np.array([dy.sum()])
    dh2 = np.outer(dy, w3)
    dz2 = dh2 * (z2 > 0)
    g_W2 = dz2.T @ h1
    g_b2 = dz2.sum(axis=0)
    dh1 = dz2 @ W2
    dz1 = dh1 * (z1 > 0)
    g_W1 = dz1.T @ X
    g_b1 = dz1.sum(axis=0)
    return np.concatenate([g_W1.ravel(), g_b1, g_W2.ravel(), g_b2, g_w3, g_b3])


def adam_step(theta, g, m, v, step, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
    m = b1 * m + (1 - b1) * g
    v = b2 * v + (1 - b2) * g * g
    mh = m / (1 - b1 ** step)
    vh = v / (1 - b2 ** step)
    return theta - lr * mh / (np.sqrt(vh) + eps), m, v
