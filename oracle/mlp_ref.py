"""FP64 CPU reference of the library's MLP cost model (test infrastructure).

y = w3 . tanh(W2 tanh(W1 x + b1) + b2) + b3, parameters packed as
W1[H][D] b1[H] W2[H][H] b2[H] w3[H] b3.  Loss: mean squared error.  The
analytic gradient below is pinned by central finite differences in the tests.
"""
import numpy as np


def num_params(D, H):
    return H * D + H + H * H + H + H + 1


def unpack(p, D, H):
    p = np.asarray(p, dtype=np.float64)
    k = 0
    W1 = p[k:k + H * D].reshape(H, D); k += H * D
    b1 = p[k:k + H]; k += H
    W2 = p[k:k + H * H].reshape(H, H); k += H * H
    b2 = p[k:k + H]; k += H
    w3 = p[k:k + H]; k += H
    b3 = p[k]
    return W1, b1, W2, b2, w3, b3


def forward(p, X, D, H):
    W1, b1, W2, b2, w3, b3 = unpack(p, D, H)
    a1 = np.tanh(np.asarray(X, np.float64) @ W1.T + b1)
    a2 = np.tanh(a1 @ W2.T + b2)
    return a2 @ w3 + b3


def loss(p, X, y, D, H):
    r = forward(p, X, D, H) - np.asarray(y, np.float64)
    return float(np.mean(r * r))


def loss_grad(p, X, y, D, H):
    X = np.asarray(X, np.float64)
    n = X.shape[0]
    W1, b1, W2, b2, w3, b3 = unpack(p, D, H)
    a1 = np.tanh(X @ W1.T + b1)
    a2 = np.tanh(a1 @ W2.T + b2)
    r = a2 @ w3 + b3 - np.asarray(y, np.float64)
    g = 2.0 * r / n
    dz2 = (g[:, None] * w3[None, :]) * (1 - a2 * a2)
    dz1 = (dz2 @ W2) * (1 - a1 * a1)
    grad = np.concatenate([(dz1.T @ X).ravel(), dz1.sum(0), (dz2.T @ a1).ravel(), dz2.sum(0),
                           a2.T @ g, [g.sum()]])
    return float(np.mean(r * r)), grad


def fd_grad(p, X, y, D, H, h=1e-6):
    p = np.asarray(p, np.float64)
    out = np.zeros_like(p)
    for k in range(p.size):
        e = np.zeros_like(p)
        e[k] = h
        out[k] = (loss(p + e, X, y, D, H) - loss(p - e, X, y, D, H)) / (2 * h)
    return out


def adam(p, g, m, v, step, lr, b1=0.9, b2=0.999, eps=1e-8):
    m = b1 * m + (1 - b1) * g
    v = b2 * v + (1 - b2) * g * g
    mh = m / (1 - b1 ** step)
    vh = v / (1 - b2 ** step)
    return p - lr * mh / (np.sqrt(vh) + eps), m, v
