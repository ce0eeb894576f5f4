"""Pins for oracle/basis.py: closed-form nodes, exactness, partition of unity, FD derivatives."""
import math

import numpy as np
import pytest

from oracle.basis import gauss_legendre, gll_nodes, lagrange, lagrange_deriv


def test_gll_closed_forms():
    # GLL points: endpoints plus roots of P_p'.  P_2' = 3x; P_3' ~ 5x^2 - 1; P_4' ~ x(7x^2 - 3).
    np.testing.assert_allclose(gll_nodes(1), [-1, 1], atol=0)
    np.testing.assert_allclose(gll_nodes(2), [-1, 0, 1], atol=0)
    s = 1 / math.sqrt(5)
    np.testing.assert_allclose(gll_nodes(3), [-1, -s, s, 1], rtol=0, atol=1e-15)
    t = math.sqrt(3 / 7)
    np.testing.assert_allclose(gll_nodes(4), [-1, -t, 0, t, 1], rtol=0, atol=1e-15)
    # p = 5: roots of P_5', x^2 = (7 -+ 2 sqrt 7)/21
    a = math.sqrt((7 - 2 * math.sqrt(7)) / 21)
    b = math.sqrt((7 + 2 * math.sqrt(7)) / 21)
    np.testing.assert_allclose(gll_nodes(5), [-1, -b, -a, a, b, 1], rtol=0, atol=1e-15)


def test_gauss_closed_forms():
    x, w = gauss_legendre(2)
    np.testing.assert_allclose(x, [-1 / math.sqrt(3), 1 / math.sqrt(3)], atol=1e-15)
    np.testing.assert_allclose(w, [1, 1], atol=1e-15)
    x, w = gauss_legendre(3)
    np.testing.assert_allclose(x, [-math.sqrt(0.6), 0, math.sqrt(0.6)], atol=1e-15)
    np.testing.assert_allclose(w, [5 / 9, 8 / 9, 5 / 9], atol=1e-15)


@pytest.mark.parametrize("n", [1, 2, 3, 5, 7])
def test_gauss_exactness(n):
    x, w = gauss_legendre(n)
    for m in range(2 * n):
        exact = 0.0 if m % 2 else 2.0 / (m + 1)
        assert abs(np.sum(w * x ** m) - exact) < 1e-14
    # degree 2n is not integrated exactly (n-point rule)
    assert abs(np.sum(w * x ** (2 * n)) - 2.0 / (2 * n + 1)) > 1e-6


@pytest.mark.parametrize("p", [1, 2, 3, 4, 5, 6])
def test_lagrange_properties(p):
    z = gll_nodes(p)
    np.testing.assert_allclose(lagrange(z, z), np.eye(p + 1), atol=1e-14)
    xs = np.linspace(-1, 1, 37)
    np.testing.assert_allclose(lagrange(z, xs).sum(axis=0), 1.0, atol=1e-13)
    np.testing.assert_allclose(lagrange_deriv(z, xs).sum(axis=0), 0.0, atol=1e-11)
    # derivative against central finite differences of the values
    h = 1e-6
    fd = (lagrange(z, xs + h) - lagrange(z, xs - h)) / (2 * h)
    np.testing.assert_allclose(lagrange_deriv(z, xs), fd, atol=1e-7)
    # the interpolant of x^p is exact
    np.testing.assert_allclose(z ** p @ lagrange(z, xs), xs ** p, atol=1e-13)
