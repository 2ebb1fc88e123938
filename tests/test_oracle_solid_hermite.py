"""Pins of the oracle's building blocks: real solid-harmonic coefficients C^a_{lm}
(Section 2, definition of H), the Hermite expansion coefficients E (recursions after
Eq. cart2herm-2) and the contraction normalisation."""
import math

import numpy as np
import pytest
from numpy.polynomial import hermite as H

import oracle


def cart(l):
    return [(l - i, i - j, j) for i in range(l + 1) for j in range(i + 1)]


def gh_moment(n, npts=40):
    """int x^n exp(-x^2) dx by Gauss-Hermite quadrature."""
    x, w = H.hermgauss(npts)
    return float(np.sum(w * x ** n))


@pytest.mark.parametrize("l", range(0, 8))
def test_solid_harmonics_are_harmonic(l):
    # the Cartesian polynomial sum_a C^a_lm x^ax y^ay z^az satisfies Laplace's equation
    C = oracle.solid_coefs(l)
    comps = cart(l)
    for row in C:
        lap = {}
        for c, (ax, ay, az) in zip(row, comps):
            for d, (k, n) in enumerate([(0, ax), (1, ay), (2, az)]):
                if n >= 2:
                    e = [ax, ay, az]
                    e[k] -= 2
                    lap[tuple(e)] = lap.get(tuple(e), 0.0) + c * n * (n - 1)
        assert max([abs(v) for v in lap.values()] + [0.0]) < 1e-12 * max(1.0, np.abs(row).max())


@pytest.mark.parametrize("l", range(0, 8))
def test_solid_harmonics_orthonormal(l):
    # overlaps of the x^l-normalised Cartesians from Gauss-Hermite moments, unit exponent
    comps = cart(l)
    S = np.zeros((len(comps), len(comps)))
    for i, a in enumerate(comps):
        for j, b in enumerate(comps):
            S[i, j] = np.prod([gh_moment(a[k] + b[k]) for k in range(3)])
    S /= S[0, 0]  # component 0 is x^l, the normalisation reference
    C = oracle.solid_coefs(l)
    assert C.shape == (2 * l + 1, len(comps))
    assert np.allclose(C @ S @ C.T, np.eye(2 * l + 1), atol=1e-12)


@pytest.mark.parametrize("l", range(1, 8))
def test_solid_harmonic_m_convention(l):
    # S_{l,m}(R_z(alpha) r) = cos(m alpha) S_lm(r) - sin(m alpha) S_{l,-m}(r) for m > 0,
    # and S_{l,|m|} has a positive x^|m| z^(l-|m|) coefficient, S_{l,-|m|} a positive
    # x^(|m|-1) y z^(l-|m|) one; m is ordered -l..l
    C = oracle.solid_coefs(l)
    comps = cart(l)
    rng = np.random.default_rng(1)
    r = rng.normal(size=(5, 3))
    alpha = 0.37
    Rz = np.array([[math.cos(alpha), -math.sin(alpha), 0], [math.sin(alpha), math.cos(alpha), 0], [0, 0, 1]])

    def val(row, pts):
        return sum(c * pts[:, 0] ** a * pts[:, 1] ** b * pts[:, 2] ** cc for c, (a, b, cc) in zip(row, comps))

    rr = r @ Rz.T
    for m in range(1, l + 1):
        p, n = C[l + m], C[l - m]
        assert np.allclose(val(p, rr), math.cos(m * alpha) * val(p, r) - math.sin(m * alpha) * val(n, r), atol=1e-12)
        assert np.allclose(val(n, rr), math.sin(m * alpha) * val(p, r) + math.cos(m * alpha) * val(n, r), atol=1e-12)
        assert p[comps.index((m, 0, l - m))] > 0
        assert n[comps.index((m - 1, 1, l - m))] > 0
    assert C[l][comps.index((0, 0, l))] > 0


@pytest.mark.parametrize("la,lb", [(0, 0), (1, 0), (2, 3), (4, 4), (6, 6), (5, 2), (7, 7), (3, 7)])
def test_hermite_expansion_reproduces_product(la, lb):
    # (x-A)^i (x-B)^j exp(-za (x-A)^2 - zb (x-B)^2)
    #   = exp(-mu AB^2) sum_t E^t_ij  d^t/dP^t exp(-zp (x-P)^2),
    # with d^t/dP^t exp(-zp (x-P)^2) = zp^(t/2) H_t(sqrt(zp)(x-P)) exp(-zp (x-P)^2)
    za, zb, A, B = 0.7, 1.9, 0.3, -0.45
    zp = za + zb
    P = (za * A + zb * B) / zp
    mu = za * zb / zp
    E = oracle.hermite_E(la, lb, za, zb, A, B)
    x = np.linspace(-2.0, 2.0, 41)
    g = np.exp(-zp * (x - P) ** 2)
    for i in range(la + 1):
        for j in range(lb + 1):
            lhs = (x - A) ** i * (x - B) ** j * np.exp(-za * (x - A) ** 2 - zb * (x - B) ** 2)
            rhs = np.zeros_like(x)
            for t in range(i + j + 1):
                c = np.zeros(t + 1)
                c[t] = 1.0
                rhs += E[i, j, t] * zp ** (t / 2) * H.hermval(math.sqrt(zp) * (x - P), c) * g
            rhs *= math.exp(-mu * (A - B) ** 2)
            assert np.allclose(lhs, rhs, atol=1e-12 * (1 + np.abs(lhs).max()))
            # coefficients beyond t = i + j vanish
            assert np.all(E[i, j, i + j + 1:] == 0)


@pytest.mark.parametrize("l,K", [(0, 1), (0, 3), (2, 2), (4, 5), (6, 3), (7, 4)])
def test_contraction_normalisation(l, K):
    # the normalised contracted x^l exp(-zeta r^2) has unit self-overlap (Gauss-Hermite)
    rng = np.random.default_rng(l * 10 + K)
    z = np.exp(rng.uniform(np.log(0.05), np.log(50), K))
    c = 1.0 - rng.uniform(0, 1, K)
    cn = oracle.contract_norm(l, z, c)
    x, w = H.hermgauss(60)
    tot = 0.0
    for i in range(K):
        for j in range(K):
            s = z[i] + z[j]
            # int x^(2l) e^{-s x^2} dx * (int e^{-s y^2} dy)^2, via x = u / sqrt(s)
            ix = np.sum(w * x ** (2 * l)) / s ** (l + 0.5)
            iy = np.sum(w) / math.sqrt(s)
            tot += cn[i] * cn[j] * ix * iy * iy
    assert tot == pytest.approx(1.0, rel=1e-12)
