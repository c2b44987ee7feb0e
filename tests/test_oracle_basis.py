"""Pins of the oracle's 1-D bases and quadrature against closed forms.

Section 3.2.1 fixes Lagrange elements on GLL nodes with tensor Gauss
quadrature; the rules themselves are textbook objects, pinned here by their
closed forms (tests/golden/quadrature_closed_forms.txt) and their exactness
degrees.
"""
import math
import os

import numpy as np
import pytest

from oracle import basis

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "quadrature_closed_forms.txt")


def _golden():
    rules = {}
    with open(GOLDEN) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            kind, n, x, w = line.split()
            rules.setdefault((kind, int(n)), []).append(
                (eval(x, {"math": math}), eval(w, {"math": math})))
    return rules


@pytest.mark.parametrize("key", sorted(_golden().keys()))
def test_rules_match_closed_forms(key):
    kind, n = key
    ref = np.array(sorted(_golden()[key]))
    x, w = basis.gauss_legendre(n) if kind == "gauss" else basis.gauss_lobatto(n)
    np.testing.assert_allclose(x, ref[:, 0], rtol=0, atol=1e-15)
    np.testing.assert_allclose(w, ref[:, 1], rtol=0, atol=2e-15)


@pytest.mark.parametrize("q", range(1, 9))
def test_gauss_exactness_degree(q):
    x, w = basis.gauss_legendre(q)
    for d in range(2 * q):
        exact = 2.0 / (d + 1) if d % 2 == 0 else 0.0
        assert abs(np.sum(w * x ** d) - exact) < 1e-14
    d = 2 * q  # first degree that is not integrated exactly
    assert abs(np.sum(w * x ** d) - 2.0 / (d + 1)) > 1e-6


@pytest.mark.parametrize("n1", range(2, 9))
def test_lobatto_exactness_degree(n1):
    x, w = basis.gauss_lobatto(n1)
    assert x[0] == -1.0 and x[-1] == 1.0
    for d in range(2 * n1 - 2):
        exact = 2.0 / (d + 1) if d % 2 == 0 else 0.0
        assert abs(np.sum(w * x ** d) - exact) < 1e-14
    d = 2 * n1 - 2
    assert abs(np.sum(w * x ** d) - 2.0 / (d + 1)) > 1e-6


@pytest.mark.parametrize("n1", range(2, 7))
def test_lagrange_kronecker_unity_and_derivatives(n1):
    xi, _ = basis.gauss_lobatto(n1)
    np.testing.assert_allclose(basis.lagrange(xi, xi), np.eye(n1), atol=1e-14)
    t = np.linspace(-1, 1, 37)
    np.testing.assert_allclose(basis.lagrange(xi, t).sum(axis=1), 1.0, atol=1e-13)
    np.testing.assert_allclose(basis.lagrange_deriv(xi, t).sum(axis=1), 0.0, atol=1e-12)
    # interpolation and differentiation are exact on polynomials of degree <= k
    for m in range(n1):
        f = xi ** m
        np.testing.assert_allclose(basis.lagrange(xi, t) @ f, t ** m, atol=1e-13)
        df = m * t ** (m - 1) if m > 0 else 0 * t
        np.testing.assert_allclose(basis.lagrange_deriv(xi, t) @ f, df, atol=1e-12)


def test_legendre_orthogonality():
    x, w = basis.gauss_legendre(12)
    for m in range(8):
        for n in range(8):
            v = np.sum(w * basis.legendre(m, x)[0] * basis.legendre(n, x)[0])
            ref = 2.0 / (2 * n + 1) if m == n else 0.0
            assert abs(v - ref) < 1e-14
    # derivative against a finite-difference-free closed form: P_3' = (15 x^2 - 3) / 2
    t = np.linspace(-1, 1, 11)
    np.testing.assert_allclose(basis.legendre(3, t)[1], (15 * t ** 2 - 3) / 2, atol=1e-13)


@pytest.mark.parametrize("k", [2, 3, 4, 5])
def test_pressure_space_dimensions(k):
    assert basis.n_pressure(k, "P") == k * (k + 1) * (k + 2) // 6
    assert basis.n_pressure(k, "Q") == (k - 1) ** 3
    # P_{k-1} modes are exactly the monomial degrees a + b + c <= k - 1
    assert all(sum(m) <= k - 1 for m in basis.pressure_modes(k, "P"))
