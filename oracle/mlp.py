"""FP64 numpy oracle of the selector network (test infrastructure only).

Network: x -> relu(W1 x + b1) -> relu(W2 . + b2) -> W3 . + b3, parameters
packed as W1 [H x F], b1 [H], W2 [H x H], b2 [H], W3 [O x H], b3 [O].  Loss:
masked mean squared error sum M (Y - T)^2 / sum M.  The gradient is derived
by the chain rule written out below; `fd_gradient` gives central finite
differences of the same loss, against which the analytic gradient is pinned.
Adam follows Kingma & Ba (ICLR 2015), bias-corrected.
"""
import numpy as np


def unpack(p, F, H, O):
    p = np.asarray(p, dtype=np.float64)
    k = 0
    out = []
    for shape in ((H, F), (H,), (H, H), (H,), (O, H), (O,)):
        size = int(np.prod(shape))
        out.append(p[k:k + size].reshape(shape))
        k += size
    assert k == p.size
    return out


def forward(p, F, H, O, X):
    W1, b1, W2, b2, W3, b3 = unpack(p, F, H, O)
    X = np.asarray(X, dtype=np.float64)
    Z1 = X @ W1.T + b1
    A1 = np.maximum(Z1, 0.0)
    Z2 = A1 @ W2.T + b2
    A2 = np.maximum(Z2, 0.0)
    Y = A2 @ W3.T + b3
    return Y, (X, Z1, A1, Z2, A2)


def loss(p, F, H, O, X, T, M):
    Y, _ = forward(p, F, H, O, X)
    M = np.asarray(M, dtype=np.float64)
    return float(np.sum(M * (Y - T) ** 2) / np.sum(M))


def gradient(p, F, H, O, X, T, M):
    W1, b1, W2, b2, W3, b3 = unpack(p, F, H, O)
    Y, (X, Z1, A1, Z2, A2) = forward(p, F, H, O, X)
    M = np.asarray(M, dtype=np.float64)
    dY = 2.0 * M * (Y - T) / np.sum(M)
    gW3 = dY.T @ A2
    gb3 = dY.sum(0)
    dZ2 = (dY @ W3) * (Z2 > 0)
    gW2 = dZ2.T @ A1
    gb2 = dZ2.sum(0)
    dZ1 = (dZ2 @ W2) * (Z1 > 0)
    gW1 = dZ1.T @ X
    gb1 = dZ1.sum(0)
    return np.concatenate([g.ravel() for g in (gW1, gb1, gW2, gb2, gW3, gb3)])


def fd_gradient(p, F, H, O, X, T, M, h=1e-6, idx=None):
    p = np.asarray(p, dtype=np.float64).copy()
    idx = range(p.size) if idx is None else idx
    g = {}
    for k in idx:
        old = p[k]
        p[k] = old + h
        lp = loss(p, F, H, O, X, T, M)
        p[k] = old - h
        lm = loss(p, F, H, O, X, T, M)
        p[k] = old
        g[k] = (lp - lm) / (2 * h)
    return g


def adam_step(p, g, m, v, t, lr, b1=0.9, b2=0.999, eps=1e-8):
    m = b1 * m + (1 - b1) * g
    v = b2 * v + (1 - b2) * g * g
    p = p - lr * (m / (1 - b1 ** t)) / (np.sqrt(v / (1 - b2 ** t)) + eps)
    return p, m, v
