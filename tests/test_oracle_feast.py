"""Pins for the oracle's FEAST loop (Algorithm 1) on one slice.

Eigenvalues are checked against NumPy's dense eigensolver and the closed-form
2-D Laplacian spectrum; eigenvector subspaces against dense eigenvectors; the
complex path against the unitary diagonal similarity D B D^H of a real band
(same eigenvalues, eigenvectors D x); counts against inertia; residuals,
orthogonality (Orth of Section 4) and the warm-start effect of Section 3
(previous eigenvectors as start vectors converge in fewer iterations).
"""
import numpy as np
import pytest

import oracle
import synth


def _slice(ab, k0, k1):
    lo = oracle.boundary_between(ab, k0)
    hi = oracle.boundary_between(ab, k1)
    return lo, hi


@pytest.mark.parametrize("cplx", [False, True])
def test_feast_random_band_matches_dense(cplx):
    n, b = 300, 7
    ab = synth.random_band(n, b, 21, cplx)
    ev, V = np.linalg.eigh(synth.band_to_dense(ab))
    lo, hi = _slice(ab, 120, 150)
    m0 = oracle.m0_rule(30)
    Y0 = synth.random_subspace(n, m0, 22, cplx)
    r = oracle.feast_slice(ab, lo, hi, Y0, ne=8, tol=1e-10)
    assert r["status"] == 0 and r["count"] == 30 and r["nfound"] == 30
    k = r["nfound"]
    bn = r["bnorm"]
    assert abs(bn - np.max(np.abs(ev))) < 1e-10
    assert np.max(np.abs(r["evals"][:k] - ev[120:150])) <= 1e-10 * bn
    X = r["evecs"][:, :k]
    assert np.max(oracle.residuals(ab, r["evals"][:k], X, bn)) <= 1e-10
    assert oracle.orth(X) < 1e-14
    assert oracle.subspace_sin_angle(X, V[:, 120:150]) < 1e-8


def test_feast_laplacian_closed_form():
    m, k = 26, 17
    ab = synth.laplacian_2d_band(m, k)
    i = np.arange(1, m + 1)[:, None]
    j = np.arange(1, k + 1)[None, :]
    ev = np.sort((4 - 2 * np.cos(i * np.pi / (m + 1)) - 2 * np.cos(j * np.pi / (k + 1))).ravel())
    lo = 0.5 * (ev[99] + ev[100])
    hi = 0.5 * (ev[139] + ev[140])
    cnt = oracle.inertia(ab, hi) - oracle.inertia(ab, lo)
    assert cnt == 40
    Y0 = synth.random_subspace(m * k, oracle.m0_rule(cnt), 5, False)
    r = oracle.feast_slice(ab, lo, hi, Y0, ne=16, rho=1.0, tol=1e-11, bnorm=float(ev[-1]))
    assert r["status"] == 0 and r["nfound"] == 40
    assert np.max(np.abs(r["evals"][:40] - ev[100:140])) < 1e-11 * ev[-1]


def test_feast_complex_phase_similarity():
    n, b = 240, 6
    ab = synth.random_band(n, b, 41)
    ph = synth.unitary_phases(n, 42)
    abz = synth.phase_similarity(ab, ph)
    lo, hi = _slice(ab, 60, 85)
    m0 = oracle.m0_rule(25)
    r0 = oracle.feast_slice(ab, lo, hi, synth.random_subspace(n, m0, 43, False), tol=1e-11)
    r1 = oracle.feast_slice(abz, lo, hi, synth.random_subspace(n, m0, 43, True), tol=1e-11)
    assert r0["status"] == 0 and r1["status"] == 0
    assert r0["nfound"] == r1["nfound"] == 25
    assert np.max(np.abs(r0["evals"][:25] - r1["evals"][:25])) < 1e-11 * r0["bnorm"]
    X0 = ph[:, None] * r0["evecs"][:, :25]
    assert oracle.subspace_sin_angle(X0, r1["evecs"][:, :25]) < 1e-8


def test_feast_counts_and_ordering():
    n, b = 200, 5
    ab = synth.random_band(n, b, 51, True)
    lo, hi = _slice(ab, 10, 22)
    r = oracle.feast_slice(ab, lo, hi, synth.random_subspace(n, 22, 52, True), tol=1e-10)
    k = r["nfound"]
    assert k == r["count"] == 12
    e = r["evals"]
    assert np.all(np.diff(e[:k]) >= 0) and np.all((e[:k] >= lo) & (e[:k] < hi))
    assert np.all((e[k:] < lo) | (e[k:] >= hi))


def test_feast_warm_start_fewer_iterations():
    # Section 3: eigenvectors of the previous matrix of an SCF-like sequence are better
    # start vectors than random ones (Table 3).
    n, b = 320, 8
    ab0 = synth.random_band(n, b, 61, True)
    ab1 = ab0 + 1e-4 * synth.perturbation(n, b, 62, True)
    lo, hi = _slice(ab1, 100, 130)
    m0 = oracle.m0_rule(30)
    cold = oracle.feast_slice(ab1, lo, hi, synth.random_subspace(n, m0, 63, True), tol=1e-10)
    prev = oracle.feast_slice(ab0, lo, hi, synth.random_subspace(n, m0, 64, True), tol=1e-10)
    warm = oracle.feast_slice(ab1, lo, hi, prev["evecs"], tol=1e-10)
    assert cold["status"] == warm["status"] == 0
    assert warm["iters"] < cold["iters"]


def test_feast_too_small_subspace_does_not_converge():
    n, b = 150, 4
    ab = synth.random_band(n, b, 71)
    lo, hi = _slice(ab, 40, 70)
    r = oracle.feast_slice(ab, lo, hi, synth.random_subspace(n, 20, 72, False), max_iter=4)
    assert r["status"] == 1 and r["nfound"] < 30


def test_m0_rule_golden():
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "m0_rule.txt")
    for line in open(path):
        if line.startswith("#") or not line.strip():
            continue
        m, expect = map(int, line.split())
        assert oracle.m0_rule(m) == expect
