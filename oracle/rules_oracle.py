"""Alternative quadrature rules for the FEAST filter -- TEST INFRASTRUCTURE (oracle).

Only ``tests/`` may import this module.  ``trapezoid_rule`` is the midpoint trapezoid rule
on the upper half of the ellipse around [lo, hi] (Section 2.2 names the trapezoid rule of
Sakurai and Sugiura beside Gauss quadrature): the Cauchy integral (1/(2 pi i)) of
dz / (z - x) over z(t) = c + r (cos t + i rho sin t), t in [0, 2 pi), with the lower half
folded onto the upper half by conjugate symmetry, and the half-turn [0, pi] split into ne
equal steps sampled at their midpoints.  ``zolotarev_rule`` is the rational filter built on
Zolotarev's best approximation of the sign function that Section 2.2 cites (after eq. (10)) as an
improvement on both; its construction is stated above the function.
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


# ----------------------------------------------------------------------------- Zolotarev rule
# Section 2.2 cites an improved rational filter built on Zolotarev's best approximation of the
# sign function (Guettel, Polizzi, Tang and Viaud, 2015) beside the Gauss and trapezoid rules.
# The construction below follows the mathematics of that approximation:
#   * Zolotarev's function of type (2m-1, 2m), the best uniform rational approximation of sign(x)
#     on [-1, -ell] U [ell, 1]:
#         s(x) = M x prod_{j=1}^{m-1} (x^2 + c_{2j}) / prod_{j=1}^{m} (x^2 + c_{2j-1}),
#         c_i = ell^2 sn^2(i K'/(2m); ell') / cn^2(i K'/(2m); ell'),  ell' = sqrt(1 - ell^2),
#     K' = K(ell'); its error 1 - s equioscillates on [ell, 1] at x_k = ell / dn(k K'/(2m); ell'),
#     k = 0..2m, and M makes the extreme errors equal in size;
#   * the Moebius map u = (lambda - lo)/(hi - lambda), x = sqrt(ell) u, which sends the slice to
#     x > 0 and the rest of the real line to x < 0; with sqrt(ell) = gap/(1 + gap) every real lambda
#     at least gap (hi - lo) away from lo and from hi lands in [-1, -ell] U [ell, 1];
#   * the filter f(lambda) = (1 + s(x(lambda)))/2; its 2m poles x = +-i sqrt(c_{2j-1}) map onto the
#     circle with diameter [lo, hi], the m in the upper half plane are the nodes z_j and the
#     weights are w_j = -Res f(z_j), so that 2 Re sum_j w_j/(z_j - lambda) = f(lambda) - f(inf).
#     The constant f(inf) = (1 - s(sqrt(ell)))/2 has size E/2 (sqrt(ell) is an equioscillation
#     point) and is dropped: a rule is nodes and weights only.  The filter is then within E of the
#     indicator of [lo, hi] outside the two transition bands.
# Elliptic functions: the arithmetic-geometric mean method (Abramowitz and Stegun 16.4 for sn, cn,
# dn; 17.6 for K), started from the complementary modulus itself so that ell' close to 1 loses no
# digits to forming 1 - ell'^2.


def agm_scale(k, kc, tol=1e-17):
    """a_n, c_n of the AGM scale started at a_0 = 1, b_0 = kc, c_0 = k (A&S 16.4.2)."""
    a, b, c = [1.0], [float(kc)], [float(k)]
    while abs(c[-1]) > tol * a[-1] and len(a) < 64:
        an = 0.5 * (a[-1] + b[-1])
        bn = np.sqrt(a[-1] * b[-1])
        cn = c[-1] * c[-1] / (4.0 * an)               # = (a_{n-1} - b_{n-1}) / 2 without cancellation
        a.append(an); b.append(bn); c.append(cn)
    return a, c


def ellip_k(kc):
    """Complete elliptic integral K of the modulus whose complement is kc: pi / (2 AGM(1, kc))."""
    k = np.sqrt(max(0.0, 1.0 - kc * kc))
    a, _ = agm_scale(k, kc)
    return np.pi / (2.0 * a[-1])


def jacobi_sn_cn_dn(u, k, kc):
    """sn, cn, dn(u; k), kc the complementary modulus: phi_N = 2^N a_N u, then
    phi_{n-1} = (phi_n + asin((c_n/a_n) sin phi_n)) / 2 (A&S 16.4.3), sn = sin phi_0,
    cn = cos phi_0, dn = sqrt(kc^2 + k^2 cn^2)."""
    a, c = agm_scale(k, kc)
    n = len(a) - 1
    phi = [0.0] * (n + 1)
    phi[n] = (2.0 ** n) * a[n] * u
    for i in range(n, 0, -1):
        phi[i - 1] = 0.5 * (phi[i] + np.arcsin(c[i] / a[i] * np.sin(phi[i])))
    sn, cn = np.sin(phi[0]), np.cos(phi[0])
    dn = np.sqrt(kc * kc + k * k * cn * cn)            # dn^2 = 1 - k^2 sn^2, both terms >= 0
    return sn, cn, dn


def zolotarev_coefficients(m, ell):
    """c_1..c_{2m-1}, M and the equioscillation error E of Zolotarev's type (2m-1, 2m) function."""
    kp = np.sqrt((1.0 - ell) * (1.0 + ell))          # ell' (modulus); ell is its complement
    Kp = ellip_k(ell)
    c = np.empty(2 * m - 1)
    for i in range(1, 2 * m):
        sn, cn, _ = jacobi_sn_cn_dn(i * Kp / (2 * m), kp, ell)
        c[i - 1] = ell * ell * sn * sn / (cn * cn)
    x1 = ell / jacobi_sn_cn_dn(Kp / (2 * m), kp, ell)[2]
    s0 = zolotarev_sign(ell, c, 1.0)
    s1 = zolotarev_sign(x1, c, 1.0)
    M = 2.0 / (s0 + s1)
    return c, M, abs(1.0 - M * s0)


def zolotarev_sign(x, c, M):
    """M x prod (x^2 + c_{2j}) / prod (x^2 + c_{2j-1}) (c indexed from c_1 at c[0])."""
    x = np.asarray(x, dtype=np.result_type(x, float))
    num = M * x
    den = np.ones_like(x)
    for i, ci in enumerate(c):
        if i % 2 == 0:
            den = den * (x * x + ci)
        else:
            num = num * (x * x + ci)
    return num / den


def zolotarev_ell(gap):
    """sqrt(ell) = gap / (1 + gap)."""
    q = gap / (1.0 + gap)
    return q * q


def zolotarev_filter(lam, lo, hi, gap, ne):
    """f(lambda) - f(inf) evaluated from the product form (the function the rule represents)."""
    ell = zolotarev_ell(gap)
    c, M, _ = zolotarev_coefficients(ne, ell)
    lam = np.asarray(lam, dtype=float)
    with np.errstate(divide="ignore", invalid="ignore"):
        x = np.sqrt(ell) * (lam - lo) / (hi - lam)
        s = np.where(lam == hi, 0.0, zolotarev_sign(x, c, M))   # x = inf at hi, where s = 0
    f = 0.5 * (1.0 + s)
    f_inf = 0.5 * (1.0 - zolotarev_sign(np.sqrt(ell), c, M))
    return f - f_inf


def zolotarev_rule(ne, lo, hi, gap):
    """Nodes z_j and weights w_j (j = 1..ne, ascending real part) of the Zolotarev filter for
    [lo, hi] with relative transition half-width gap, and the bound E on |filter - indicator|
    outside the bands within gap (hi - lo) of lo and of hi."""
    m = ne
    ell = zolotarev_ell(gap)
    c, M, E = zolotarev_coefficients(m, ell)
    odd, even = c[0::2], c[1::2]                      # c_1, c_3, ... and c_2, c_4, ...
    sq = np.sqrt(ell)
    z = np.empty(m, dtype=np.complex128)
    w = np.empty(m, dtype=np.complex128)
    for j in range(m):
        xj = 1j * np.sqrt(odd[j])                     # pole of s in the upper half plane
        # residue of s at xj: M P(-c_{2j-1}) / (2 prod_{k != j} (c_{2k-1} - c_{2j-1}))
        res_s = M * np.prod(even - odd[j]) / (2.0 * np.prod(np.delete(odd, j) - odd[j]))
        u = xj / sq
        z[j] = (lo + hi * u) / (1.0 + u)
        dlam_dx = (hi - lo) / (sq * (1.0 + u) ** 2)
        w[j] = -0.5 * res_s * dlam_dx                 # -Res of f = (1 + s)/2 at z_j
    return z, w, E
