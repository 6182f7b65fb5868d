"""Alternative quadrature rule for the FEAST filter -- TEST INFRASTRUCTURE (oracle).

Only ``tests/`` may import this module.  ``trapezoid_rule`` is the midpoint trapezoid rule
on the upper half of the ellipse around [lo, hi] (Section 2.2 names the trapezoid rule of
Sakurai and Sugiura beside Gauss quadrature): the Cauchy integral (1/(2 pi i)) of
dz / (z - x) over z(t) = c + r (cos t + i rho sin t), t in [0, 2 pi), with the lower half
folded onto the upper half by conjugate symmetry, and the half-turn [0, pi] split into ne
equal steps sampled at their midpoints.
"""
import numpy as np


def trapezoid_rule(ne, lo, hi, rho=0.3):
    c = 0.5 * (lo + hi)
    r = 0.5 * (hi - lo)
    t = np.pi * (np.arange(ne) + 0.5) / ne
    z = c + r * (np.cos(t) + 1j * rho * np.sin(t))
    dz = r * (-np.sin(t) + 1j * rho * np.cos(t))        # z'(t)
    w = dz * (np.pi / ne) / (2j * np.pi)                 # (1/(2 pi i)) z'(t) dt
    return z, w


def filter_value(z, w, x):
    """r(x) = 2 Re sum_k w_k / (z_k - x): the lower half of the contour is the conjugate."""
    return float(2.0 * np.real(np.sum(w / (z - x))))
