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


# ----------------------------------------------------------------------------- Zolotarev rule
# The rational filter Section 2.2 cites after eq. (10) as an improvement on the Gauss and
# trapezoid rules, built on Zolotarev's best approximation of sign(x).  The pins: the elliptic
# functions against an independent library and their special values; the m = 1 function in closed
# form; Chebyshev equioscillation (which characterises the unique best approximation) found on a
# dense grid without the oracle's own extremum formula; the partial fractions (nodes and weights)
# against the product form; the indicator bound; FEAST convergence with the rule.

@pytest.mark.parametrize("ell", [0.3, 0.6, 0.9])
def test_oracle_elliptic_functions(ell):
    from scipy.special import ellipj, ellipkm1
    kp = np.sqrt(1.0 - ell * ell)
    K = ro.ellip_k(ell)                               # K of modulus kp
    assert abs(K - ellipkm1(ell * ell)) <= 4e-16 * K
    for u in (0.0, 0.13, 0.5 * K, 0.77 * K, K, 1.6 * K):
        sn, cn, dn = ro.jacobi_sn_cn_dn(u, kp, ell)
        rs, rc, rd, _ = ellipj(u, kp * kp)
        assert abs(sn - rs) < 1e-14 and abs(cn - rc) < 1e-14 and abs(dn - rd) < 1e-14
    sn, cn, dn = ro.jacobi_sn_cn_dn(K, kp, ell)
    assert abs(sn - 1.0) < 1e-15 and abs(cn) < 1e-15 and abs(dn - ell) < 1e-15
    sn, cn, dn = ro.jacobi_sn_cn_dn(0.5 * K, kp, ell)       # half period: dn = sqrt(kc), sn^2 = 1/(1+kc)
    assert abs(dn - np.sqrt(ell)) < 1e-15 and abs(sn * sn - 1.0 / (1.0 + ell)) < 1e-15


def test_oracle_elliptic_functions_small_complement():
    """ell' = sqrt(1 - ell^2) near 1: K ~ ln(4/ell), and the identities hold without the loss of
    digits that forming 1 - ell'^2 would cause.  At u = K/2 the amplitude sits sqrt(ell) below
    pi/2, so the rounding of u itself (about eps K) moves dn = cn-scaled values by eps K/sqrt(ell)
    relatively: the tolerance is that conditioning, 8e-15/sqrt(ell)."""
    from scipy.special import ellipkm1
    for ell in (1e-2, 1e-4, 1e-6):
        K = ro.ellip_k(ell)
        assert abs(K - ellipkm1(ell * ell)) <= 1e-15 * K
        kp = np.sqrt((1.0 - ell) * (1.0 + ell))
        sn, cn, dn = ro.jacobi_sn_cn_dn(0.5 * K, kp, ell)
        assert abs(dn / np.sqrt(ell) - 1.0) < 8e-15 / np.sqrt(ell)
        assert abs(sn * sn + cn * cn - 1.0) < 1e-15 and abs(dn * dn + kp * kp * sn * sn - 1.0) < 1e-15


@pytest.mark.parametrize("ell", [0.5, 0.05, 0.003])
def test_zolotarev_m1_closed_form(ell):
    """m = 1: c_1 = ell (sc^2(K'/2; ell') = 1/ell), s(x) = M x/(x^2 + ell) with extrema of the error
    at ell, sqrt(ell), 1: M = 2 / (1/(1+ell) + 1/(2 sqrt(ell))), E = 1 - M/(1+ell).  The rule is one
    node at the top of the circle with diameter [lo, hi], weight i M r / (4 sqrt(ell))."""
    c, M, E = ro.zolotarev_coefficients(1, ell)
    rel = 1e-14 / np.sqrt(ell)                        # conditioning of sc, dn at K'/2 (see above)
    assert abs(c[0] - ell) <= rel * ell
    Mc = 2.0 / (1.0 / (1.0 + ell) + 1.0 / (2.0 * np.sqrt(ell)))
    assert abs(M - Mc) <= rel * Mc and abs(E - (1.0 - Mc / (1.0 + ell))) <= rel
    lo, hi = -0.7, 2.3
    gap = np.sqrt(ell) / (1.0 - np.sqrt(ell))         # the gap whose sqrt(ell) = gap/(1+gap) is this one
    z, w, E2 = ro.zolotarev_rule(1, lo, hi, gap)
    r = 0.5 * (hi - lo)
    assert abs(z[0] - complex(0.5 * (lo + hi), r)) <= rel * r
    wc = 1j * Mc * r / (4.0 * np.sqrt(ell))
    assert abs(w[0] - wc) <= rel * abs(wc) and abs(E2 - E) < 1e-13


@pytest.mark.parametrize("m", [2, 3, 5, 8])
@pytest.mark.parametrize("ell", [0.3, 0.02, 0.002])
def test_zolotarev_equioscillation(m, ell):
    """The error 1 - s(x) on [ell, 1] alternates in sign across 2m+1 runs of a dense grid and
    reaches the same magnitude E in every run: by Chebyshev's alternation theorem s is then the
    best approximation of type (2m-1, 2m) (odd), which is unique.  E shrinks as m grows."""
    c, M, E = ro.zolotarev_coefficients(m, ell)
    if E < 1e-9:
        pytest.skip("error below what a grid in double precision resolves")
    x = np.geomspace(ell, 1.0, 400001)
    e = 1.0 - ro.zolotarev_sign(x, c, M)
    sign = np.sign(e)
    cut = np.flatnonzero(sign[1:] != sign[:-1]) + 1
    runs = np.split(e, cut)
    assert len(runs) == 2 * m + 1
    peaks = np.array([r[np.argmax(np.abs(r))] for r in runs])
    assert np.all(np.sign(peaks[1:]) == -np.sign(peaks[:-1]))
    assert np.max(np.abs(np.abs(peaks) / E - 1.0)) < 1e-6
    assert ro.zolotarev_coefficients(m + 1, ell)[2] < E
    # odd symmetry and the reflection x -> ell/x that maps [ell, 1] onto itself
    xs = np.array([0.37, 1.9, 11.0]) * np.sqrt(ell)
    assert np.allclose(ro.zolotarev_sign(-xs, c, M), -ro.zolotarev_sign(xs, c, M), rtol=1e-14, atol=0)
    assert np.allclose(ro.zolotarev_sign(ell / xs, c, M), ro.zolotarev_sign(xs, c, M), rtol=1e-12, atol=0)


@pytest.mark.parametrize("ne,gap", [(1, 0.2), (2, 0.05), (5, 0.1), (8, 0.05), (8, 0.3), (12, 0.02)])
def test_zolotarev_rule_filter(ne, gap):
    """Nodes and weights against the product form of the filter (a dropped term, a wrong residue
    sign or a wrong map shows here), the bound E outside the transition bands, the values 1/2 - f_inf
    at lo and hi, mirror symmetry about the centre, nodes on the circle over [lo, hi]."""
    lo, hi = 2.0, 3.5
    c, r = 0.5 * (lo + hi), 0.5 * (hi - lo)
    z, w, E = ro.zolotarev_rule(ne, lo, hi, gap)
    assert np.all(z.imag > 0) and np.all(np.diff(z.real) > 0)
    assert np.max(np.abs(np.abs(z - c) - r)) < 1e-14
    lam = np.concatenate([np.linspace(-10.0, 15.0, 2001), lo + (hi - lo) * np.array([1e-9, 0.3, 0.5, 1 - 1e-9])])
    rule = np.array([ro.filter_value(z, w, x) for x in lam])
    assert np.max(np.abs(rule - ro.zolotarev_filter(lam, lo, hi, gap, ne))) < 1e-13
    d = np.minimum(np.abs(lam - lo), np.abs(lam - hi))
    far = d >= gap * (hi - lo)
    ind = ((lam >= lo) & (lam <= hi)).astype(float)
    assert np.max(np.abs(rule[far] - ind[far])) <= E + 1e-13      # 1e-13: rounding of the sum
    f_inf = 0.5 - ro.filter_value(z, w, lo)
    assert abs(ro.filter_value(z, w, hi) - (0.5 - f_inf)) < 1e-13
    assert abs(abs(f_inf) - 0.5 * E) < 1e-13
    # the oracle computes every c_i directly, so the mirror pairs of nodes carry the conditioning
    # of sc near K' (about eps K'/sqrt(ell) relative): 1e-12 covers gap >= 0.02
    for t in (0.1, 0.45, 0.9, 1.3, 4.0):
        assert abs(ro.filter_value(z, w, c + r * t) - ro.filter_value(z, w, c - r * t)) < 1e-12
    # the bands are sharp: just inside them the bound no longer holds once E is small
    if E < 1e-3:
        assert abs(ro.filter_value(z, w, lo - 0.02 * gap * (hi - lo))) > 10 * E


def test_zolotarev_rule_oracle_feast():
    """The oracle's FEAST (Algorithm 1) converges with the Zolotarev rule to the exact counts."""
    import oracle
    import synth
    n, b = 400, 8
    ab = synth.random_band(n, b, 501, True)
    ks = [100, 140, 175]
    bounds = [oracle.boundary_between(ab, k) for k in ks]
    bn = oracle.spectral_norm(ab)
    m0 = [oracle.m0_rule(40), oracle.m0_rule(35)]
    X0 = synth.random_subspace(n, sum(m0), 502, True)
    ev = np.linalg.eigvalsh(synth.band_to_dense(ab))
    off = 0
    for i in range(2):
        z, w, _ = ro.zolotarev_rule(8, bounds[i], bounds[i + 1], 0.1)
        cnt = ks[i + 1] - ks[i]
        o = oracle.feast_slice(ab, bounds[i], bounds[i + 1], X0[:, off:off + m0[i]], tol=1e-10, bnorm=bn,
                               max_iter=40, count=cnt, rule=(z, w))
        assert o["status"] == 0 and o["nfound"] == cnt and o["iters"] <= 6
        assert np.max(np.abs(o["evals"][:cnt] - ev[ks[i]:ks[i + 1]])) <= 1e-10 * bn
        off += m0[i]


@pytest.mark.parametrize("ne", [1, 2, 5, 8, 16])
@pytest.mark.parametrize("gap", [0.05, 0.2, 1.0, 2.3, 2.5, 40.0])
def test_library_zolotarev_rule_matches_oracle(ne, gap):
    """gap 2.3 / 2.5 sit on both sides of ell = 1/2, where the library switches from the nome series
    of sn/cn to the amplitude recursion (the oracle uses the recursion throughout)."""
    import paper_2012_00506_gb300 as pk
    from paper_2012_00506_gb300 import build
    build.build()
    lo, hi = -0.7, 2.3
    z, w, E = pk.zolotarev_rule(ne, lo, hi, gap)
    zo, wo, Eo = ro.zolotarev_rule(ne, lo, hi, gap)
    assert np.max(np.abs(z - zo)) <= 1e-12 * max(abs(lo), abs(hi))
    assert np.max(np.abs(w - wo)) <= 1e-12 * np.max(np.abs(wo))
    assert abs(E - Eo) <= 1e-9 * Eo + 1e-14          # E = |1 - M s(ell)| carries absolute rounding


def test_library_zolotarev_rule_arguments():
    """Argument errors come back as the documented negative codes; large ne stays finite."""
    import ctypes as C
    import paper_2012_00506_gb300 as pk
    from paper_2012_00506_gb300 import build
    build.build()
    lib = pk.load()
    z = np.zeros(300, dtype=np.complex128)
    w = np.zeros(300, dtype=np.complex128)
    pz, pw = z.ctypes.data_as(C.c_void_p), w.ctypes.data_as(C.c_void_p)
    f = lib.pdeshep_contour_rule_zolotarev
    assert f(0, 0.0, 1.0, 0.1, pz, pw, None) == -1 and f(257, 0.0, 1.0, 0.1, pz, pw, None) == -1
    assert f(4, 1.0, 1.0, 0.1, pz, pw, None) == -2 and f(4, 0.0, float("inf"), 0.1, pz, pw, None) == -2
    assert f(4, 0.0, 1.0, 0.0, pz, pw, None) == -4 and f(4, 0.0, 1.0, float("nan"), pz, pw, None) == -4
    assert f(4, 0.0, 1.0, 0.9e-8, pz, pw, None) == -4 and f(4, 0.0, 1.0, 1e-8, pz, pw, None) == 0
    assert f(4, 0.0, 1.0, 0.1, None, pw, None) == -5 and f(4, 0.0, 1.0, 0.1, pz, None, None) == -6
    assert f(256, 0.0, 1.0, 0.01, pz, pw, None) == 0
    assert np.all(np.isfinite(z[:256])) and np.all(np.isfinite(w[:256]))
    for x, want in ((-0.5, 0.0), (0.25, 1.0), (0.75, 1.0), (1.5, 0.0)):
        assert abs(2.0 * np.real(np.sum(w[:256] / (z[:256] - x))) - want) < 1e-11


@pytest.mark.parametrize("ne", [1, 4, 16, 64, 128, 256])
@pytest.mark.parametrize("gap", [1e-8, 1e-6, 1e-4, 0.05, 1.0, 2.3, 2.5, 1e6])
def test_library_zolotarev_rule_accuracy_over_its_domain(ne, gap):
    """Across the accepted parameters the library's filter stays within E + delta of the indicator
    outside the transition bands, delta the documented rounding floor (1e-12 for gap >= 1e-4,
    1e-10 for gap >= 1e-6, 1e-9 below), nodes and weights finite, nodes in the upper half plane --
    also on a slice near the top of the double range."""
    import paper_2012_00506_gb300 as pk
    from paper_2012_00506_gb300 import build
    build.build()
    for lo, hi in ((-1.0, 1.0), (-1e307, 1e307)):
        z, w, E = pk.zolotarev_rule(ne, lo, hi, gap)
        assert np.all(np.isfinite(z)) and np.all(np.isfinite(w)) and np.all(z.imag > 0)
    z, w, E = pk.zolotarev_rule(ne, -1.0, 1.0, gap)
    delta = 1e-12 if gap >= 1e-4 else (1e-10 if gap >= 1e-6 else 1e-9)
    d = 2.0 * gap                                      # gap (hi - lo)
    t = np.linspace(0.0, 30.0, 60)
    xs = list(1 + d * (1 + t)) + list(-1 - d * (1 + t))
    if d < 1:
        xs += list(np.linspace(-1 + d, 1 - d, 61))
    for x in xs:
        want = 1.0 if -1.0 < x < 1.0 else 0.0
        assert abs(2.0 * np.real(np.sum(w / (z - x))) - want) <= E + delta
