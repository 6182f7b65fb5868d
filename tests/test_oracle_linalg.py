"""Pins for the oracle's shifted band LU/solves (eq. (10)), band product, CholQR and
Jacobi eigensolver (Rayleigh-Ritz of Section 2.2).

References are LAPACK through NumPy/SciPy on dense expansions (getrf uses the
same first-maximum |Re|+|Im| pivot rule, so pivot indices must agree exactly)
and mathematical invariants.
"""
import numpy as np
import pytest
import scipy.linalg as sl

import oracle
import synth


@pytest.mark.parametrize("n,b,cplx,z", [
    (1, 0, False, 0.3 + 0.2j), (2, 1, True, -0.1 + 0.01j), (9, 3, False, 0.05 + 0.001j),
    (50, 7, True, 0.2 + 0.03j), (131, 12, False, -0.4 + 0.1j), (64, 16, True, 0.0 + 1e-4j),
    (40, 45, True, 0.5 + 0.5j)])
def test_band_lu_matches_lapack(n, b, cplx, z):
    ab = synth.random_band(n, b, 31 + n, cplx)
    A = synth.band_to_dense(ab)
    M = z * np.eye(n) - A
    F, ipiv, info = oracle.band_lu(ab, z)
    assert info == 0
    lu, piv = sl.lu_factor(M)
    assert np.array_equal(piv, ipiv)
    # U lives in rows k..k+2b of the LAPACK band layout: F[j, 2b + i - j] = U[i, j]
    U = np.triu(lu)
    for j in range(n):
        for i in range(max(0, j - 2 * b), j + 1):
            assert abs(F[j, 2 * b + i - j] - U[i, j]) <= 1e-12 * max(1.0, abs(U[i, j]))
    Y = synth.random_subspace(n, 5, 2, True)
    for trans in (0, 1):
        X = oracle.band_solve(F, ipiv, b, Y, trans)
        ref = np.linalg.solve(M if trans == 0 else M.conj().T, Y)
        assert np.max(np.abs(X - ref)) <= 1e-10 * np.max(np.abs(ref))
        Mt = M if trans == 0 else M.conj().T
        assert np.linalg.norm(Mt @ X - Y) <= 1e-13 * np.linalg.norm(Mt) * np.linalg.norm(X)


def test_band_lu_zero_matrix_is_scaled_identity():
    n, b = 20, 3
    ab = np.zeros((n, b + 1))
    z = 0.7 - 0.2j
    F, ipiv, info = oracle.band_lu(ab, z)
    assert info == 0 and np.array_equal(ipiv, np.arange(n))
    Y = synth.random_subspace(n, 3, 5, True)
    assert np.allclose(oracle.band_solve(F, ipiv, b, Y, 0), Y / z, atol=1e-15)
    assert np.allclose(oracle.band_solve(F, ipiv, b, Y, 1), Y / np.conj(z), atol=1e-15)


def test_band_lu_reports_singular():
    ab = synth.diagonal_band([1.0, 0.0, 2.0], 1)
    _, _, info = oracle.band_lu(ab, 0.0)
    assert info == 2


@pytest.mark.parametrize("cplx", [False, True])
def test_band_matvec_matches_dense(cplx):
    n, b = 77, 6
    ab = synth.random_band(n, b, 9, cplx)
    X = synth.random_subspace(n, 4, 10, True)
    assert np.allclose(oracle.band_matvec(ab, X), synth.band_to_dense(ab) @ X, atol=1e-14)


@pytest.mark.parametrize("cplx", [False, True])
def test_cholqr(cplx):
    n, m = 200, 17
    Q0 = synth.random_subspace(n, m, 4, cplx)
    Q, R, info = oracle.cholqr(Q0)
    assert info == 0
    assert np.allclose(np.triu(R), R) and np.all(np.real(np.diag(R)) > 0)
    assert np.allclose(np.imag(np.diag(R)), 0)
    assert np.linalg.norm(Q @ R - Q0) < 1e-13 * np.linalg.norm(Q0)
    assert np.max(np.abs(Q.conj().T @ Q - np.eye(m))) < 1e-13
    Qr, Rr = np.linalg.qr(np.asarray(Q0, dtype=np.complex128))
    ph = np.diag(Rr) / np.abs(np.diag(Rr))
    assert np.allclose(R, (Rr.T * ph.conj()).T, atol=1e-12)


def test_cholqr_breakdown():
    Q0 = np.ones((10, 3))
    _, _, info = oracle.cholqr(Q0)
    assert info >= 2


@pytest.mark.parametrize("m,cplx", [(1, False), (2, True), (10, False), (37, True), (64, False)])
def test_jacobi_matches_eigh(m, cplx):
    rng = np.random.default_rng(m)
    A = rng.normal(size=(m, m))
    if cplx:
        A = A + 1j * rng.normal(size=(m, m))
    A = 0.5 * (A + A.conj().T)
    lam, V, sweeps = oracle.jacobi_eig(A)
    assert sweeps >= 0
    ref = np.linalg.eigvalsh(A)
    assert np.max(np.abs(lam - ref)) < 1e-13 * max(1.0, np.linalg.norm(A))
    assert np.max(np.abs(V.conj().T @ V - np.eye(m))) < 1e-13
    assert np.linalg.norm(A @ V - V * lam) < 1e-12 * max(1.0, np.linalg.norm(A))
    for j in range(m):  # phase convention: largest component real positive
        k = np.argmax(np.abs(V[:, j]))
        assert V[k, j].real > 0 and V[k, j].imag == 0


def test_jacobi_degenerate():
    m = 12
    rng = np.random.default_rng(3)
    U, _ = np.linalg.qr(rng.normal(size=(m, m)) + 1j * rng.normal(size=(m, m)))
    d = np.array([1.0] * 4 + [2.0] * 5 + [-3.0] * 3)
    A = (U * d) @ U.conj().T
    lam, V, _ = oracle.jacobi_eig(A)
    assert np.allclose(lam, np.sort(d), atol=1e-13)
    assert np.max(np.abs(V.conj().T @ V - np.eye(m))) < 1e-13
    assert np.linalg.norm(A @ V - V * lam) < 1e-12
