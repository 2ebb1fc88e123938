"""Pins of the oracle's Coulomb/exchange digestion (oracle.jk) against facts fixed by the
mathematics, not by its own formula:

* a one-hot density reduces J to one (. . | lam sig) slice of the integral block and K to one
  (. nu | . sig) slice, which fixes where every index goes (a transposed or swapped index
  fails);
* a single (ss|ss) quartet of normalised s Gaussians has a closed form;
* over every shell 4-tuple of a small basis, both "energies" are squared norms in the
  Coulomb metric and so non-negative for any real D:
      sum D_mn J_mn = int int rho(1) rho(2) / r12 >= 0,  rho(r) = sum D_mn phi_m phi_n,
      sum D_ml K_ml = int int g(1,2)^2 / r12 >= 0,       g(1,2) = sum D_ml phi_m(1) phi_l(2),
  and J, K are symmetric for symmetric D."""
import itertools
import math

import numpy as np
import pytest

import oracle

from test_oracle_eri import make_basis


def small_basis(ls=(1, 0, 2), seed=3):
    rng = np.random.default_rng(seed)
    centers = rng.uniform(0, 1.5, (len(ls), 3))
    exps = [np.exp(rng.uniform(np.log(0.3), np.log(3.0), 2)) for _ in ls]
    coefs = [1.0 - rng.uniform(0, 1, 2) for _ in ls]
    return make_basis(list(ls), centers, exps, coefs)


@pytest.mark.parametrize("solid", [False, True])
def test_one_hot_density_selects_integral_slices(solid):
    b = small_basis((2, 1, 3, 1))
    q = [[0, 1, 2, 3]]
    bf, nbf = oracle.function_offsets(b, solid)
    n = [2 * l + 1 if solid else (l + 1) * (l + 2) // 2 for l in (2, 1, 3, 1)]
    out, _ = oracle.eri(b, q, solid=solid)
    I = out.reshape(n)
    rng = np.random.default_rng(0)
    for _ in range(3):
        lam, sig, nu = rng.integers(n[2]), rng.integers(n[3]), rng.integers(n[1])
        D = np.zeros((nbf, nbf))
        D[bf[2] + lam, bf[3] + sig] = 1.0
        J, K = oracle.jk(b, q, D, solid)
        assert np.array_equal(J[bf[0]:bf[0] + n[0], bf[1]:bf[1] + n[1]], I[:, :, lam, sig])
        D = np.zeros((nbf, nbf))
        D[bf[1] + nu, bf[3] + sig] = 1.0
        J, K = oracle.jk(b, q, D, solid)
        assert np.array_equal(K[bf[0]:bf[0] + n[0], bf[2]:bf[2] + n[2]], I[:, nu, :, sig])
        # nothing lands outside the quartet's blocks
        mask = np.zeros_like(K, bool)
        mask[bf[0]:bf[0] + n[0], bf[2]:bf[2] + n[2]] = True
        assert not K[~mask].any()


def test_ssss_closed_form():
    # (ss|ss) of normalised single Gaussians: 2 pi^(5/2) / (p q sqrt(p+q)) exp(-ab/p AB^2 - cd/q CD^2)
    # F0(pq/(p+q) PQ^2) times the four normalisations (2z/pi)^(3/4)
    z = [0.9, 1.7, 0.5, 2.2]
    C = np.array([[0.0, 0.0, 0.0], [0.4, -0.2, 0.3], [1.1, 0.5, -0.6], [0.7, 0.9, 0.2]])
    b = make_basis([0, 0, 0, 0], C, [[x] for x in z])
    p, q = z[0] + z[1], z[2] + z[3]
    P, Q = (z[0] * C[0] + z[1] * C[1]) / p, (z[2] * C[2] + z[3] * C[3]) / q
    T = p * q / (p + q) * np.sum((P - Q) ** 2)
    F0 = 0.5 * math.sqrt(math.pi / T) * math.erf(math.sqrt(T))
    ref = (2 * math.pi ** 2.5 / (p * q * math.sqrt(p + q)) * F0 *
           math.exp(-z[0] * z[1] / p * np.sum((C[0] - C[1]) ** 2) - z[2] * z[3] / q * np.sum((C[2] - C[3]) ** 2)) *
           np.prod([(2 * x / math.pi) ** 0.75 for x in z]))
    D = np.arange(16.0).reshape(4, 4) / 7.0
    J, K = oracle.jk(b, [[0, 1, 2, 3]], D)
    assert J[0, 1] == pytest.approx(ref * D[2, 3], rel=1e-13)
    assert K[0, 2] == pytest.approx(ref * D[1, 3], rel=1e-13)
    assert np.count_nonzero(J) == 1 and np.count_nonzero(K) == 1


@pytest.mark.parametrize("solid", [False, True])
def test_full_list_energies_nonnegative_and_symmetric(solid):
    b = small_basis()
    q = list(itertools.product(range(3), repeat=4))
    _, nbf = oracle.function_offsets(b, solid)
    rng = np.random.default_rng(1)
    for sym in (True, False):
        D = rng.standard_normal((nbf, nbf))
        if sym:
            D = D + D.T
        J, K = oracle.jk(b, q, D, solid)
        scale = np.abs(J).max() * np.abs(D).max() * nbf
        assert np.sum(D * J) >= -1e-12 * scale
        assert np.sum(D * K) >= -1e-12 * scale
        if sym:
            assert np.abs(J - J.T).max() <= 1e-13 * np.abs(J).max()
            assert np.abs(K - K.T).max() <= 1e-13 * np.abs(K).max()
