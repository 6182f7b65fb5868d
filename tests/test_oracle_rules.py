"""The midpoint trapezoid rule on the half ellipse (Section 2.2 names it beside Gauss
quadrature): oracle pins from closed forms, and the library's rule against the oracle."""
import numpy as np
import pytest

from oracle import rules_oracle as ro


@pytest.mark.parametrize("ne", [4, 8, 16])
def test_circle_filter_closed_form(ne):
    """On a circle the 2 ne midpoint nodes are the roots of z^(2ne) = -1 around c, and the filter
    is 1 / (1 + t^(2ne)), t = (x - c)/r, for real x: 1/2 at the interval ends, 1 at the centre."""
    lo, hi = -0.7, 1.9
    c, r = 0.5 * (lo + hi), 0.5 * (hi - lo)
    z, w = ro.trapezoid_rule(ne, lo, hi, rho=1.0)
    for t in (0.0, 0.3, -0.8, 1.0, -1.0, 1.2, -2.5, 4.0):
        assert abs(ro.filter_value(z, w, c + r * t) - 1.0 / (1.0 + t ** (2 * ne))) < 2e-14


def test_ellipse_filter_converges_to_the_indicator():
    lo, hi = 2.0, 3.0
    c, r = 2.5, 0.5
    for rho in (0.3, 0.6):
        z, w = ro.trapezoid_rule(128, lo, hi, rho)
        for t in (0.0, 0.4, -0.7):
            assert abs(ro.filter_value(z, w, c + r * t) - 1.0) < 1e-6
        for t in (1.4, -1.6, 3.0):
            assert abs(ro.filter_value(z, w, c + r * t)) < 1e-6
        # mirror symmetry of the node set about the vertical axis through c
        z8, w8 = ro.trapezoid_rule(8, lo, hi, rho)
        for t in (0.2, 0.9, 1.7):
            assert abs(ro.filter_value(z8, w8, c + r * t) - ro.filter_value(z8, w8, c - r * t)) < 1e-13


@pytest.mark.parametrize("ne,lo,hi,rho", [(1, -1.0, 1.0, 0.3), (8, -0.7, -0.2, 0.3), (16, 2.0, 9.0, 1.0)])
def test_library_trapezoid_rule_matches_oracle(ne, lo, hi, rho):
    import paper_2012_00506_gb300 as pk
    from paper_2012_00506_gb300 import build
    build.build()
    z, w = pk.contour_rule(ne, lo, hi, rho, kind="trapezoid")
    zo, wo = ro.trapezoid_rule(ne, lo, hi, rho)
    scale = max(1.0, abs(lo), abs(hi))
    assert np.max(np.abs(z - zo)) <= 4e-16 * scale * 4
    assert np.max(np.abs(w - wo)) <= 4e-16 * scale * 4
