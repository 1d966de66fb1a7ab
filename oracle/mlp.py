"""Oracle for the selector's cost model (test infrastructure only).

FP64 numpy restatement of the network the library's CUDA kernels train:
    h1 = relu(W1 x + b1),  h2 = relu(W2 h1 + b2),  y = W3 h2 + b3,
    loss = sum_{r,k} m_rk (y_rk - t_rk)^2 / sum m,
its gradient by the chain rule, and one bias-corrected Adam step.  Parameters
are one flat vector laid out W1 (H x IN, row-major), b1, W2, b2, W3, b3.  The
paper fixes no model (model-based selection is its future work), so the pins
are mathematical: finite differences, closed forms, special cases.
"""
import numpy as np

IN, H, OUT = 10, 64, 8      # inputs: op one-hot [3], log2 n, log2 batch, mode one-hot [5]
NPARAM = H * IN + H + H * H + H + OUT * H + OUT


def unpack(p):
    p = np.asarray(p, dtype=np.float64)
    o = 0
    def take(k, shape):
        nonlocal o
        v = p[o:o + k].reshape(shape)
        o += k
        return v
    W1 = take(H * IN, (H, IN)); b1 = take(H, (H,))
    W2 = take(H * H, (H, H)); b2 = take(H, (H,))
    W3 = take(OUT * H, (OUT, H)); b3 = take(OUT, (OUT,))
    return W1, b1, W2, b2, W3, b3


def pack(W1, b1, W2, b2, W3, b3):
    return np.concatenate([np.ravel(a) for a in (W1, b1, W2, b2, W3, b3)]).astype(np.float64)


def forward(p, X):
    """Returns y [rows x OUT] and the intermediates (a1, h1, a2, h2)."""
    W1, b1, W2, b2, W3, b3 = unpack(p)
    X = np.asarray(X, dtype=np.float64)
    a1 = X @ W1.T + b1
    h1 = np.maximum(a1, 0.0)
    a2 = h1 @ W2.T + b2
    h2 = np.maximum(a2, 0.0)
    y = h2 @ W3.T + b3
    return y, (a1, h1, a2, h2)


def loss(p, X, T, M):
    y, _ = forward(p, X)
    M = np.asarray(M, dtype=np.float64)
    return float((M * (y - T) ** 2).sum() / max(M.sum(), 1e-300))


def loss_and_grad(p, X, T, M):
    """Loss and its gradient (flat vector) by backpropagation."""
    W1, b1, W2, b2, W3, b3 = unpack(p)
    X = np.asarray(X, dtype=np.float64)
    M = np.asarray(M, dtype=np.float64)
    y, (a1, h1, a2, h2) = forward(p, X)
    n = max(M.sum(), 1e-300)
    L = float((M * (y - T) ** 2).sum() / n)
    dy = 2.0 * M * (y - T) / n                  # dL/dy
    gW3 = dy.T @ h2
    gb3 = dy.sum(axis=0)
    da2 = (dy @ W3) * (a2 > 0)                  # through relu
    gW2 = da2.T @ h1
    gb2 = da2.sum(axis=0)
    da1 = (da2 @ W2) * (a1 > 0)
    gW1 = da1.T @ X
    gb1 = da1.sum(axis=0)
    return L, pack(gW1, gb1, gW2, gb2, gW3, gb3)


def adam_step(p, g, m, v, step, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update (Kingma & Ba), bias-corrected; returns (p, m, v)."""
    m = beta1 * m + (1 - beta1) * g
    v = beta2 * v + (1 - beta2) * g * g
    mh = m / (1 - beta1 ** step)
    vh = v / (1 - beta2 ** step)
    return p - lr * mh / (np.sqrt(vh) + eps), m, v


def init_params(seed=0):
    """He-style random initialisation (used by tests and training)."""
    rng = np.random.default_rng(seed)
    W1 = rng.standard_normal((H, IN)) * np.sqrt(2.0 / IN)
    W2 = rng.standard_normal((H, H)) * np.sqrt(2.0 / H)
    W3 = rng.standard_normal((OUT, H)) * np.sqrt(1.0 / H)
    return pack(W1, np.zeros(H), W2, np.zeros(H), W3, np.zeros(OUT))
