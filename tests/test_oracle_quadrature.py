"""Pins for the oracle's quadrature rule (Section 2.2, eqs. (8)-(9)).

The Gauss-Legendre rule is checked against NumPy's library routine, closed-form
nodes and exactness on polynomials; the contour rule against the Cauchy
integral (indicator function of the slice) and a closed form at the centre.
"""
import numpy as np
import pytest

import oracle


@pytest.mark.parametrize("ne", [1, 2, 3, 5, 8, 12, 16, 24, 32])
def test_gauss_legendre_matches_numpy(ne):
    x, w = oracle.gauss_legendre(ne)
    xr, wr = np.polynomial.legendre.leggauss(ne)
    assert np.max(np.abs(x - xr)) < 1e-14
    assert np.max(np.abs(w - wr)) < 1e-14


def test_gauss_legendre_closed_forms():
    x, w = oracle.gauss_legendre(2)
    assert np.allclose(x, [-1 / np.sqrt(3), 1 / np.sqrt(3)], atol=1e-15, rtol=0)
    assert np.allclose(w, [1.0, 1.0], atol=1e-15, rtol=0)
    x, w = oracle.gauss_legendre(3)
    assert np.allclose(x, [-np.sqrt(0.6), 0.0, np.sqrt(0.6)], atol=1e-15, rtol=0)
    assert np.allclose(w, [5 / 9, 8 / 9, 5 / 9], atol=1e-15, rtol=0)


@pytest.mark.parametrize("ne", [4, 8, 16])
def test_gauss_legendre_polynomial_exactness(ne):
    x, w = oracle.gauss_legendre(ne)
    assert abs(w.sum() - 2.0) < 1e-14
    for k in range(2 * ne):
        exact = 2.0 / (k + 1) if k % 2 == 0 else 0.0
        assert abs(np.sum(w * x**k) - exact) < 1e-13, k
    # degree 2ne is not integrated exactly
    k = 2 * ne
    assert abs(np.sum(w * x**k) - 2.0 / (k + 1)) > 1e-12


def test_contour_rule_circle_centre_is_exactly_one():
    # rho = 1, x = c: w_k/(z_k - c) = omega_k/4, so r(c) = sum(omega)/2 = 1
    for ne in (1, 3, 8, 16):
        z, w = oracle.contour_rule(ne, -0.7, 1.9, rho=1.0)
        assert abs(oracle.filter_value(z, w, 0.6) - 1.0) < 1e-14


@pytest.mark.parametrize("rho", [0.3, 0.6, 1.0])
def test_contour_rule_converges_to_indicator(rho):
    lo, hi = 0.25, 0.75
    z, w = oracle.contour_rule(400, lo, hi, rho)
    for x in (0.3, 0.45, 0.5, 0.7):
        assert abs(oracle.filter_value(z, w, x) - 1.0) < 1e-8
    for x in (-1.0, 0.0, 0.2, 0.8, 1.0, 3.0):
        assert abs(oracle.filter_value(z, w, x)) < 1e-8


@pytest.mark.parametrize("ne", [8, 16])
def test_contour_rule_filter_shape(ne):
    lo, hi = -1.0, 1.0
    z, w = oracle.contour_rule(ne, lo, hi, 0.3)
    assert np.all(z.imag > 0)                       # upper half-plane
    assert np.all(np.abs(z - 0.0) <= 1.0 + 1e-15)    # on the ellipse inside the circle
    r = lambda x: oracle.filter_value(z, w, x)
    # symmetric about the centre (node set is symmetric under theta -> pi - theta)
    for s in (0.1, 0.5, 0.99, 1.2, 3.0):
        assert abs(r(s) - r(-s)) < 1e-13
    assert abs(r(0.0) - 1.0) < 0.1
    assert 0.3 < r(1.0) < 0.7 and 0.3 < r(-1.0) < 0.7
    assert abs(r(3.0)) < 1e-2 and abs(r(10.0)) < 1e-4
    # nodes lie on the ellipse (x-c)^2/r^2 + y^2/(rho r)^2 = 1
    assert np.allclose(z.real**2 + (z.imag / 0.3) ** 2, 1.0, atol=1e-14)


def test_contour_weights_are_cauchy_discretisation():
    # sum_k w_k/(z_k - x) is the quadrature of (1/2 pi i) int_0^pi z'(theta)/(z(theta)-x) dtheta;
    # compare one slice with a direct trapezoid evaluation of that integral on a fine grid.
    lo, hi, rho, x = 0.0, 2.0, 0.5, 0.4
    th = np.linspace(0, np.pi, 200001)
    zc = 1.0 + np.cos(th) + 1j * rho * np.sin(th)
    dz = -np.sin(th) + 1j * rho * np.cos(th)
    f = dz / (zc - x) / (2j * np.pi)
    half = np.trapezoid(f, th)
    z, w = oracle.contour_rule(64, lo, hi, rho)
    approx = np.sum(w / (z - x))
    assert abs(approx - half) < 1e-8
    assert abs(2 * half.real - 1.0) < 1e-8


@pytest.mark.parametrize("ne,rho", [(4, 0.3), (8, 0.3), (16, 0.3), (8, 0.6), (16, 1.0)])
def test_filter_at_centre_closed_form(ne, rho):
    # At x = c, 2 Re[z'(th)/(z(th)-c)]/(2 pi i) = rho / (pi (cos^2 th + rho^2 sin^2 th)); the rule is
    # Gauss-Legendre on th = (pi/2)(1 - t), so r(c) = sum_k omega_k (pi/2) rho/(pi(cos^2 + rho^2 sin^2)).
    t, om = np.polynomial.legendre.leggauss(ne)
    th = 0.5 * np.pi * (1 - t)
    expect = np.sum(om * 0.5 * rho / (np.cos(th) ** 2 + rho**2 * np.sin(th) ** 2))
    z, w = oracle.contour_rule(ne, 2.0, 5.0, rho)
    assert abs(oracle.filter_value(z, w, 3.5) - expect) < 1e-13
