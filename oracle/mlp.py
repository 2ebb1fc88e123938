"""Reference forward pass and gradient of the router MLP, in float64 numpy.

TEST INFRASTRUCTURE ONLY (part of the oracle): the GPU training kernels are checked
against it.  Network: 20 inputs -> 64 -> 64 -> NOUT = 2 outputs, ReLU, parameters packed as
W1[64][20], b1[64], W2[64][64], b2[64], W3[2][64], b3[2]; loss = the mean over samples of the
summed squared errors of the outputs, L = (1/n) sum_i sum_o (y_io - t_io)^2.  The gradient is
the plain chain rule; tests/test_oracle_mlp.py pins it to central finite differences of the
loss and to the network's affine special case.  No part of the paper corresponds to it.
"""
import numpy as np

NIN, NW, NOUT = 20, 64, 2
SIZES = [("W1", (NW, NIN)), ("b1", (NW,)), ("W2", (NW, NW)), ("b2", (NW,)), ("W3", (NOUT, NW)), ("b3", (NOUT,))]
NPARAM = sum(int(np.prod(s)) for _, s in SIZES)


def unpack(p):
    p = np.asarray(p, dtype=np.float64)
    out, o = {}, 0
    for name, shape in SIZES:
        n = int(np.prod(shape))
        out[name] = p[o:o + n].reshape(shape)
        o += n
    return out


def pack(d):
    return np.concatenate([np.asarray(d[name], dtype=np.float64).reshape(-1) for name, _ in SIZES])


def forward(p, X):
    """Outputs y (n x NOUT) and the intermediate values of the pass."""
    w = unpack(p)
    a1 = X @ w["W1"].T + w["b1"]
    h1 = np.maximum(a1, 0.0)
    a2 = h1 @ w["W2"].T + w["b2"]
    h2 = np.maximum(a2, 0.0)
    y = h2 @ w["W3"].T + w["b3"]
    return y, (X, a1, h1, a2, h2)


def loss(p, X, t):
    y, _ = forward(p, X)
    return float(np.sum((y - t) ** 2) / len(t))


def loss_and_grad(p, X, t):
    """Loss and its gradient with respect to the packed parameters (t is n x NOUT)."""
    w = unpack(p)
    y, (X, a1, h1, a2, h2) = forward(p, X)
    n = len(t)
    r = y - t
    dy = 2.0 * r / n  # n x NOUT
    g = {"W3": dy.T @ h2, "b3": dy.sum(0)}
    d2 = (dy @ w["W3"]) * (a2 > 0)
    g["W2"] = d2.T @ h1
    g["b2"] = d2.sum(0)
    d1 = (d2 @ w["W2"]) * (a1 > 0)
    g["W1"] = d1.T @ X
    g["b1"] = d1.sum(0)
    return float(np.sum(r ** 2) / n), pack(g)
