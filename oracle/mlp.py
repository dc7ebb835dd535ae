"""FP64 reference of the surrogate MLP (test infrastructure only).

The surrogate maps 33 inputs (32 circuit features and log10 p) to the
probability that a trajectory passes its success criterion:
    h1 = relu(x W1 + b1)        W1: 33 x 256
    h2 = relu(h1 W2 + b2)       W2: 256 x 256
    z  = h2 w3 + b3             w3: 256
    P  = sigmoid(z)
trained with the mean binary cross-entropy of z against 0/1 pass labels and
Adam. The GPU keeps weights in bfloat16 (FP32 master copies) and accumulates
in FP32; this reference computes in float64 on whatever (already rounded)
weights it is given.
"""
import numpy as np

SIZES = (33, 256, 256, 1)


def init_params(rng, sizes=SIZES):
    """He-uniform weights, zero biases."""
    p = {}
    for i, (a, b) in enumerate(zip(sizes[:-1], sizes[1:])):
        lim = np.sqrt(6.0 / a)
        p[f"W{i + 1}"] = rng.uniform(-lim, lim, size=(a, b))
        p[f"b{i + 1}"] = np.zeros(b)
    return p


def forward(p, x):
    h1 = np.maximum(x @ p["W1"] + p["b1"], 0.0)
    h2 = np.maximum(h1 @ p["W2"] + p["b2"], 0.0)
    z = (h2 @ p["W3"] + p["b3"])[:, 0]
    return z, (x, h1, h2)


def sigmoid(z):
    return 1.0 / (1.0 + np.exp(-z))


def bce(z, y):
    """Mean of softplus(z) - y z, i.e. -[y log s + (1 - y) log(1 - s)], s = sigmoid(z)."""
    return float(np.mean(np.logaddexp(0.0, z) - y * z))


def backward(p, cache, z, y):
    """Gradients of bce(z, y) with respect to every parameter."""
    x, h1, h2 = cache
    B = x.shape[0]
    dz = (sigmoid(z) - y) / B                     # d bce / d z
    g = {"W3": h2.T @ dz[:, None], "b3": np.array([dz.sum()])}
    dh2 = (dz[:, None] @ p["W3"].T) * (h2 > 0)
    g["W2"] = h1.T @ dh2
    g["b2"] = dh2.sum(0)
    dh1 = (dh2 @ p["W2"].T) * (h1 > 0)
    g["W1"] = x.T @ dh1
    g["b1"] = dh1.sum(0)
    return g


def adam(p, g, state, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam step (Kingma & Ba 2015) with bias correction; updates p in place."""
    state["t"] = state.get("t", 0) + 1
    t = state["t"]
    for k in p:
        m = state.setdefault("m_" + k, np.zeros_like(p[k]))
        v = state.setdefault("v_" + k, np.zeros_like(p[k]))
        m[:] = b1 * m + (1 - b1) * g[k]
        v[:] = b2 * v + (1 - b2) * g[k] ** 2
        mh = m / (1 - b1 ** t)
        vh = v / (1 - b2 ** t)
        p[k] -= lr * mh / (np.sqrt(vh) + eps)
    return p


def bf16_round(a):
    """Round float64 values to the nearest bfloat16 (ties to even), as float64."""
    f = np.asarray(a, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)
