"""Pins for the oracle's Sylvester-inertia count (Section 3.2).

Counts are checked against the closed-form spectrum of the 2-D Laplacian, the
diagonal case, and NumPy's dense eigenvalues; every pivot of the pivot-free
LDL^T is checked against ratios of leading principal minors (d_k =
det(A_{k+1}) / det(A_k)).
"""
import numpy as np
import pytest

import oracle
import synth


def _laplacian_eigs(m, k):
    i = np.arange(1, m + 1)[:, None]
    j = np.arange(1, k + 1)[None, :]
    return np.sort((4 - 2 * np.cos(i * np.pi / (m + 1)) - 2 * np.cos(j * np.pi / (k + 1))).ravel())


@pytest.mark.parametrize("m,k", [(7, 5), (20, 9), (63, 32)])
def test_laplacian_counts_closed_form(m, k):
    ab = synth.laplacian_2d_band(m, k)
    ev = _laplacian_eigs(m, k)
    u = np.unique(np.round(ev, 12))
    rng = np.random.default_rng(0)
    picks = rng.choice(len(u) - 1, size=min(12, len(u) - 1), replace=False)
    for p in picks:
        sigma = 0.5 * (u[p] + u[p + 1])
        assert oracle.inertia(ab, sigma) == int(np.sum(ev < sigma))
    assert oracle.inertia(ab, -0.1) == 0
    assert oracle.inertia(ab, 8.1) == m * k


def test_diagonal_counts_and_zero_pivot():
    d = np.array([0.5, -1.0, 2.0, -1.0, 0.0, 3.0, -2.5])
    for b in (0, 3):
        ab = synth.diagonal_band(d, b)
        for sigma in (-3.0, -1.5, 0.25, 2.5, 10.0):
            assert oracle.inertia(ab, sigma) == int(np.sum(d < sigma))
        # sigma equal to a diagonal entry: exact zero pivot counted as negative
        pm = oracle.pivmin(ab)
        cnt, piv = oracle.inertia(ab, -1.0, return_pivots=True)
        assert cnt == int(np.sum(d <= -1.0))
        assert np.sum(piv == -pm) == 2


@pytest.mark.parametrize("n,b,cplx", [(60, 1, False), (97, 7, False), (80, 12, True), (33, 40, True),
                                      (1, 0, False), (5, 4, True)])
def test_random_counts_match_dense(n, b, cplx):
    ab = synth.random_band(n, b, 100 + n + b, cplx)
    ev = np.linalg.eigvalsh(synth.band_to_dense(ab))
    for sigma in np.linspace(ev[0] - 0.1, ev[-1] + 0.1, 10):
        if np.min(np.abs(ev - sigma)) < 1e-9:
            continue
        assert oracle.inertia(ab, sigma) == int(np.sum(ev < sigma))


@pytest.mark.parametrize("cplx", [False, True])
def test_pivots_are_ratios_of_leading_minors(cplx):
    n, b = 40, 5
    ab = synth.random_band(n, b, 7, cplx)
    A = synth.band_to_dense(ab)
    sigma = 0.13
    M = A - sigma * np.eye(n)
    _, piv = oracle.inertia(ab, sigma, return_pivots=True)
    prev_sign, prev_log = 1.0, 0.0
    for k in range(n):
        s, lg = np.linalg.slogdet(M[: k + 1, : k + 1])
        s = np.real(s)
        dk = s / prev_sign * np.exp(lg - prev_log)
        assert abs(piv[k] - dk) <= 1e-9 * max(1.0, abs(dk)), k
        prev_sign, prev_log = s, lg


def test_complex_phase_similarity_same_inertia():
    n, b = 150, 9
    ab = synth.random_band(n, b, 11)
    abz = synth.phase_similarity(ab, synth.unitary_phases(n, 12))
    for sigma in (-0.7, -0.1, 0.0, 0.33, 0.9):
        c0, p0 = oracle.inertia(ab, sigma, return_pivots=True)
        c1, p1 = oracle.inertia(abz, sigma, return_pivots=True)
        assert c0 == c1
        assert np.max(np.abs(p0 - p1) / np.maximum(1.0, np.abs(p0))) < 1e-10


def test_bisection_boundaries():
    ab = synth.random_band(300, 6, 3)
    ev = np.linalg.eigvalsh(synth.band_to_dense(ab))
    for k in (1, 50, 150, 299):
        s = oracle.boundary_between(ab, k)
        assert ev[k - 1] < s < ev[k]
        assert abs(s - 0.5 * (ev[k - 1] + ev[k])) < 1e-12
    assert abs(oracle.spectral_norm(ab) - np.max(np.abs(ev))) < 1e-11
