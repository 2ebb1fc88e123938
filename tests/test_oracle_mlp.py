"""Pin of the oracle's router-MLP gradient: central finite differences of its loss."""
import numpy as np

from oracle import mlp


def test_gradient_matches_finite_differences():
    rng = np.random.default_rng(0)
    p = rng.normal(scale=0.3, size=mlp.NPARAM)
    X = rng.normal(size=(37, mlp.NIN))
    t = rng.normal(size=37)
    L, g = mlp.loss_and_grad(p, X, t)
    assert L == mlp.loss(p, X, t)
    idx = rng.choice(mlp.NPARAM, 80, replace=False)
    idx = np.concatenate([idx, [0, mlp.NPARAM - 1, mlp.NPARAM - 2]])  # include b3 and W3
    h = 1e-6
    for i in idx:
        e = np.zeros(mlp.NPARAM)
        e[i] = h
        fd = (mlp.loss(p + e, X, t) - mlp.loss(p - e, X, t)) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(g[i])), i


def test_linear_special_case():
    # with positive pre-activations everywhere the network is affine in X: the gradient of
    # b3 is the mean residual times 2, and y equals the product of the weight matrices
    rng = np.random.default_rng(1)
    w = {"W1": np.abs(rng.normal(size=(64, 20))), "b1": np.ones(64), "W2": np.abs(rng.normal(size=(64, 64))),
         "b2": np.ones(64), "W3": rng.normal(size=64), "b3": np.array([0.3])}
    p = mlp.pack(w)
    X = np.abs(rng.normal(size=(5, 20)))
    y, _ = mlp.forward(p, X)
    ref = (((X @ w["W1"].T + 1) @ w["W2"].T + 1) @ w["W3"]) + 0.3
    assert np.allclose(y, ref, rtol=1e-12)
    t = np.zeros(5)
    _, g = mlp.loss_and_grad(p, X, t)
    assert np.isclose(g[-1], 2 * np.mean(y - t))
