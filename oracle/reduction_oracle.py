"""Steps (I) and (III) of PDESHEP -- TEST INFRASTRUCTURE (oracle).

Only ``tests/`` may import this module.  Plain NumPy, FP64/complex128, following the
paper's Section 2.1 (two-step reduction, eqs. for D = U A U^H and X = U^H X_hat) and
Algorithm 2 (Step (I): block Householder transformations reduce A to a banded matrix;
Step (III): backtransform of the band's eigenvectors):

* ``dense_to_band(A, b)``   for every panel of b columns (left to right), the block
                            below the band is factored A[j+b:, j:j+b] = Q R (a library
                            QR serves as the block Householder step) and Q^H ... Q is
                            applied to the trailing rows and columns; returns the banded
                            D (dense storage, entries beyond the band set to zero) and
                            W = U^H with D = W^H A W.
* ``to_lower_band(D, b)``   LAPACK lower compact band storage (n, b + 1): ab[i, k] =
                            D[i + k, i], the layout of the band FEAST input.
* ``backtransform(W, Xh)``  X = U^H X_hat = W X_hat (Step (III)).
* ``generalized_to_standard(A, B)``  the generalized problem A x = lambda B x (A Hermitian, B
                            Hermitian positive definite) reduced to the standard one by the
                            Cholesky factor B = L L^H: A~ = L^{-1} A L^{-H} with eigenvectors
                            x~ = L^H x (Section 2.1); returns A~ and L.
* ``standard_to_generalized(L, Xt)``  x = L^{-H} x~ for every column.
"""
from __future__ import annotations

import numpy as np


def dense_to_band(A, b):
    """D, W with D = W^H A W banded (semi-bandwidth b) and W unitary."""
    A = np.array(A, copy=True)
    n = A.shape[0]
    assert A.shape == (n, n) and b >= 1
    W = np.eye(n, dtype=A.dtype)
    for j in range(0, n - b - 1, b):                # panels with at least two rows below the band
        r0 = j + b                                   # first row below the band of this panel
        Q, _ = np.linalg.qr(A[r0:, j:j + b], mode="complete")
        # two-sided update of the trailing part: rows r0: by Q^H, columns r0: by Q
        A[r0:, :] = Q.conj().T @ A[r0:, :]
        A[:, r0:] = A[:, r0:] @ Q
        W[:, r0:] = W[:, r0:] @ Q
    D = np.zeros_like(A)
    for k in range(-b, b + 1):
        idx = np.arange(max(0, -k), min(n, n - k))
        D[idx + k, idx] = A[idx + k, idx]
    D = 0.5 * (D + D.conj().T)                      # exact Hermitian symmetry of the result
    return D, W


def to_lower_band(D, b):
    n = D.shape[0]
    ab = np.zeros((n, b + 1), dtype=D.dtype)
    for k in range(b + 1):
        i = np.arange(n - k)
        ab[i, k] = D[i + k, i]
    return ab


def backtransform(W, Xh):
    return W @ Xh


def generalized_to_standard(A, B):
    """A~ = L^{-1} A L^{-H}, B = L L^H (lower Cholesky factor), A~ made exactly Hermitian."""
    L = np.linalg.cholesky(B)
    Y = np.linalg.solve(L, A)                        # L^{-1} A
    At = np.linalg.solve(L, Y.conj().T).conj().T     # (L^{-1} (L^{-1} A)^H)^H = L^{-1} A L^{-H}
    return 0.5 * (At + At.conj().T), L


def standard_to_generalized(L, Xt):
    return np.linalg.solve(L.conj().T, Xt)
