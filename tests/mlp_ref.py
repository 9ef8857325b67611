"""float64 numpy reference of the cost perceptron 16 -> 64 -> 64 -> 1 (ReLU),
written from the layer equations; test infrastructure only."""
import numpy as np

IN, H = 16, 64
W1, B1 = 0, H * IN
W2 = B1 + H
B2 = W2 + H * H
W3 = B2 + H
B3 = W3 + H
NPARAM = B3 + 1


def bf16_round(a):
    """Round float32 values to bfloat16 (nearest, ties to even), as float64."""
    a = np.asarray(a, dtype=np.float32)
    u = a.view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def unpack(p):
    p = np.asarray(p, dtype=np.float64)
    return (p[W1:B1].reshape(H, IN), p[B1:W2], p[W2:B2].reshape(H, H), p[B2:W3], p[W3:B3],
            p[B3])


def weights_bf16(p):
    """Weights rounded to bf16 (biases kept), the forward pass's parameters."""
    q = np.asarray(p, dtype=np.float64).copy()
    for lo, hi in ((W1, B1), (W2, B2), (W3, B3)):
        q[lo:hi] = bf16_round(np.asarray(p[lo:hi], dtype=np.float32))
    return q


def forward(p, x, act_bf16=False):
    w1, b1, w2, b2, w3, b3 = unpack(p)
    x = np.asarray(x, dtype=np.float64)
    if act_bf16:
        x = bf16_round(x.astype(np.float32))
    z1 = x @ w1.T + b1
    h1 = np.maximum(z1, 0)
    if act_bf16:
        h1 = bf16_round(h1.astype(np.float32))
    z2 = h1 @ w2.T + b2
    h2 = np.maximum(z2, 0)
    return h2 @ w3 + b3, (x, z1, h1, z2, h2)


def loss_grad(p, x, y):
    """Mean squared error and its gradient with respect to p."""
    w1, b1, w2, b2, w3, b3 = unpack(p)
    out, (x, z1, h1, z2, h2) = forward(p, x)
    n = x.shape[0]
    d = out - np.asarray(y, dtype=np.float64)
    loss = np.mean(d * d)
    dy = 2.0 * d / n
    g = np.zeros(NPARAM)
    g[W3:B3] = h2.T @ dy
    g[B3] = dy.sum()
    dz2 = np.outer(dy, w3) * (z2 > 0)
    g[W2:B2] = (dz2.T @ h1).ravel()
    g[B2:W3] = dz2.sum(0)
    dz1 = (dz2 @ w2) * (z1 > 0)
    g[W1:B1] = (dz1.T @ x).ravel()
    g[B1:W2] = dz1.sum(0)
    return loss, g


def adam(p, g, m, v, step, lr, b1, b2, eps):
    m = b1 * m + (1 - b1) * g
    v = b2 * v + (1 - b2) * g * g
    p = p - lr * (m / (1 - b1 ** step)) / (np.sqrt(v / (1 - b2 ** step)) + eps)
    return p, m, v


def random_params(rng):
    p = np.zeros(NPARAM)
    p[W1:B1] = rng.normal(0, np.sqrt(2 / IN), H * IN)
    p[B1:W2] = rng.normal(0, 0.1, H)
    p[W2:B2] = rng.normal(0, np.sqrt(2 / H), H * H)
    p[B2:W3] = rng.normal(0, 0.1, H)
    p[W3:B3] = rng.normal(0, np.sqrt(1 / H), H)
    p[B3] = 0.3
    return p
