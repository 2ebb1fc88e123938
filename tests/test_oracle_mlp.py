"""Pins of the oracle's router MLP: its gradient against central finite differences of its
loss, and its forward pass and output-bias gradient in the special case where the network is
affine."""
import numpy as np

from oracle import mlp


def test_gradient_matches_finite_differences():
    rng = np.random.default_rng(0)
    p = rng.normal(scale=0.3, size=mlp.NPARAM)
    X = rng.normal(size=(37, mlp.NIN))
    t = rng.normal(size=(37, mlp.NOUT))
    L, g = mlp.loss_and_grad(p, X, t)
    assert L == mlp.loss(p, X, t)
    idx = rng.choice(mlp.NPARAM, 80, replace=False)
    # include both output biases and weights of both output rows
    last = mlp.NPARAM - 1
    idx = np.concatenate([idx, [0, last, last - 1, last - 2, last - 2 - mlp.NW]])
    h = 1e-6
    for i in idx:
        e = np.zeros(mlp.NPARAM)
        e[i] = h
        fd = (mlp.loss(p + e, X, t) - mlp.loss(p - e, X, t)) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(g[i])), i


def test_linear_special_case():
    # with positive pre-activations everywhere the network is affine in X: each output equals
    # the product of the weight matrices, and the gradient of each output's bias is twice that
    # output's mean residual
    rng = np.random.default_rng(1)
    w = {"W1": np.abs(rng.normal(size=(64, 20))), "b1": np.ones(64), "W2": np.abs(rng.normal(size=(64, 64))),
         "b2": np.ones(64), "W3": rng.normal(size=(2, 64)), "b3": np.array([0.3, -0.7])}
    p = mlp.pack(w)
    X = np.abs(rng.normal(size=(5, 20)))
    y, _ = mlp.forward(p, X)
    h2 = (X @ w["W1"].T + 1) @ w["W2"].T + 1
    for o in range(2):
        assert np.allclose(y[:, o], h2 @ w["W3"][o] + w["b3"][o], rtol=1e-12)
    t = np.zeros((5, 2))
    _, g = mlp.loss_and_grad(p, X, t)
    assert np.allclose(g[-2:], 2 * np.mean(y - t, axis=0))


def test_outputs_are_independent_heads():
    # the loss separates over the outputs: changing the target of one output leaves the
    # gradient of the other output's last-layer row and bias unchanged
    rng = np.random.default_rng(2)
    p = rng.normal(scale=0.3, size=mlp.NPARAM)
    X = rng.normal(size=(11, mlp.NIN))
    t = rng.normal(size=(11, 2))
    t2 = t.copy()
    t2[:, 1] += 3.0
    _, g = mlp.loss_and_grad(p, X, t)
    _, g2 = mlp.loss_and_grad(p, X, t2)
    w3 = mlp.NPARAM - 2 - 2 * mlp.NW
    assert np.array_equal(g[w3:w3 + mlp.NW], g2[w3:w3 + mlp.NW])  # row 0 of W3
    assert g[-2] == g2[-2]  # b3[0]
    assert not np.allclose(g[w3 + mlp.NW:w3 + 2 * mlp.NW], g2[w3 + mlp.NW:w3 + 2 * mlp.NW])
