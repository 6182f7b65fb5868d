"""Pins of the Step (I)/(III) oracle (dense -> band reduction D = U A U^H by block Householder
transformations, backtransform X = U^H X_hat; Section 2.1 and Algorithm 2 of the paper) against
LAPACK eigenvalues and the defining identities."""
import numpy as np
import pytest

import synth
from oracle import reduction_oracle as ro


def _herm(n, cplx, seed):
    g = np.random.default_rng(seed)
    A = g.standard_normal((n, n)) + (1j * g.standard_normal((n, n)) if cplx else 0)
    return 0.5 * (A + A.conj().T)


@pytest.mark.parametrize("cplx", [False, True])
@pytest.mark.parametrize("n,b", [(50, 4), (37, 5), (20, 1), (64, 16), (33, 32)])
def test_reduction_identities(cplx, n, b):
    A = _herm(n, cplx, 100 + n + b)
    nrm = np.linalg.norm(A, 2)
    D, W = ro.dense_to_band(A, b)
    # W unitary, D = W^H A W exactly banded (the product recomputed here, not the oracle's D)
    assert np.max(np.abs(W.conj().T @ W - np.eye(n))) < 1e-14 * n
    F = W.conj().T @ A @ W
    for k in range(b + 1, n):
        assert np.max(np.abs(np.diag(F, -k))) < 1e-14 * nrm * n
    assert np.max(np.abs(F - D)) < 1e-14 * nrm * n
    # same spectrum as A (LAPACK)
    assert np.max(np.abs(np.linalg.eigvalsh(D) - np.linalg.eigvalsh(A))) < 1e-13 * nrm
    # Step (III): eigenvectors of the band mapped back are eigenvectors of A
    lam, Xh = np.linalg.eigh(D)
    X = ro.backtransform(W, Xh)
    assert np.max(np.linalg.norm(A @ X - X * lam, axis=0)) < 1e-13 * nrm * np.sqrt(n)
    # band storage is the FEAST input layout
    assert np.array_equal(synth.band_to_dense(ro.to_lower_band(D, b)), D)


def test_reduction_trivial_bandwidth():
    A = _herm(12, True, 7)
    D, W = ro.dense_to_band(A, 11)
    assert np.array_equal(W, np.eye(12)) and np.array_equal(D, 0.5 * (A + A.conj().T))


def _spd(n, cplx, seed):
    g = np.random.default_rng(seed)
    G = g.standard_normal((n, n)) + (1j * g.standard_normal((n, n)) if cplx else 0)
    return G @ G.conj().T / n + np.eye(n)


@pytest.mark.parametrize("cplx", [False, True])
@pytest.mark.parametrize("n", [1, 7, 60])
def test_generalized_to_standard_against_library(cplx, n):
    """The pencil's eigenvalues from SciPy's generalized solver; the eigenvectors mapped back by
    x = L^{-H} x~ are B-orthonormal and satisfy A x = lambda B x."""
    from scipy.linalg import eigh
    A = _herm(n, cplx, 300 + n)
    B = _spd(n, cplx, 400 + n)
    At, L = ro.generalized_to_standard(A, B)
    assert np.max(np.abs(L @ L.conj().T - B)) <= 1e-14 * np.linalg.norm(B, 2) * n
    assert np.max(np.abs(np.triu(L, 1))) == 0
    lam, Xt = np.linalg.eigh(At)
    ref = eigh(A, B, eigvals_only=True)
    nrm = np.max(np.abs(ref))
    assert np.max(np.abs(lam - ref)) <= 1e-13 * nrm * max(n, 1)
    X = ro.standard_to_generalized(L, Xt)
    assert np.max(np.abs(X.conj().T @ B @ X - np.eye(n))) <= 1e-13 * n
    assert np.max(np.linalg.norm(A @ X - (B @ X) * lam, axis=0)) <= 1e-12 * nrm * n


def test_generalized_to_standard_special_cases():
    """B = I leaves A and gives L = I; B diagonal gives A~ = D^{-1/2} A D^{-1/2}, L = D^{1/2}."""
    A = _herm(9, True, 5)
    At, L = ro.generalized_to_standard(A, np.eye(9))
    assert np.array_equal(L, np.eye(9)) and np.max(np.abs(At - A)) == 0
    d = np.linspace(0.5, 4.0, 9)
    At, L = ro.generalized_to_standard(A, np.diag(d))
    assert np.max(np.abs(L - np.diag(np.sqrt(d)))) <= 1e-15 * 2
    assert np.max(np.abs(At - A / np.sqrt(np.outer(d, d)))) <= 1e-15 * np.max(np.abs(A)) * 4
