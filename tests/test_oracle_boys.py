"""Pins of the oracle's Boys function F_m(T) = int_0^1 y^{2m} exp(-T y^2) dy (Eq. boys)."""
import math

import numpy as np
import pytest
from scipy import special

import oracle

TS = [0.0, 1e-10, 1e-4, 0.05, 0.5, 1.0, 3.3, 7.0, 12.5, 20.0, 33.0, 47.0, 60.0, 79.99, 80.01, 95.0, 150.0, 400.0,
      2500.0, 4.0e4]


def test_zero_argument():
    # F_m(0) = 1/(2m+1)
    F = oracle.boys(40, 0.0)
    assert np.allclose(F, 1.0 / (2 * np.arange(41) + 1), rtol=1e-15, atol=0)


@pytest.mark.parametrize("T", [t for t in TS if t > 0])
def test_f0_is_error_function(T):
    # F_0(T) = sqrt(pi / (4T)) erf(sqrt T)
    ref = math.sqrt(math.pi / (4 * T)) * math.erf(math.sqrt(T))
    assert oracle.boys(0, T)[0] == pytest.approx(ref, rel=2e-15)


@pytest.mark.parametrize("T", [t for t in TS if t > 0])
def test_incomplete_gamma(T):
    # F_m(T) = gamma(m + 1/2, T) / (2 T^(m + 1/2)) (the integral with y^2 = s/T)
    m = np.arange(0, 33)
    a = m + 0.5
    P = special.gammainc(a, T)
    ok = P > 1e-280  # the regularised gamma underflows for tiny T at high m
    ref = np.exp(np.log(P[ok]) + special.gammaln(a[ok]) - a[ok] * np.log(T)) / 2.0
    F = oracle.boys(32, T)[ok]
    assert ok.sum() >= 10
    assert np.allclose(F, ref, rtol=2e-13, atol=0)


@pytest.mark.parametrize("T", [0.3, 9.0, 40.0, 200.0])
def test_definition_by_quadrature(T):
    # the defining integral by adaptive quadrature
    for m in (0, 1, 5, 12, 24):
        val, err = __import__("scipy.integrate", fromlist=["quad"]).quad(
            lambda y: y ** (2 * m) * math.exp(-T * y * y), 0.0, 1.0, epsabs=0.0, epsrel=1e-13, limit=200)
        assert oracle.boys(m, T)[m] == pytest.approx(val, rel=1e-12)


@pytest.mark.parametrize("T", [t for t in TS if t > 0])
def test_recursion_identity(T):
    # integration by parts: 2T F_{m+1}(T) = (2m+1) F_m(T) - exp(-T), for every m
    F = oracle.boys(30, T)
    m = np.arange(30)
    lhs = 2 * T * F[1:]
    rhs = (2 * m + 1) * F[:-1] - math.exp(-T)
    # the right side cancels for small T; its rounding is ~eps * (2m+1) F_m
    tol = 1e-12 * np.abs(lhs) + 4e-16 * (2 * m + 1) * F[:-1]
    assert np.all(np.abs(lhs - rhs) <= tol)


def test_branch_continuity():
    # the series branch (T <= 80) and the erf + upward branch (T > 80) meet smoothly
    a = oracle.boys(28, 80.0)
    b = oracle.boys(28, 80.0 + 1e-9)
    assert np.allclose(a, b, rtol=1e-9)


def test_monotone_and_positive():
    for T in TS:
        F = oracle.boys(24, T)
        assert np.all(F > 0)
        assert np.all(np.diff(F) < 0)
