"""Pins for the oracle's metric helpers that every parity test leans on.

* ``subspace_sin_angle``: the sine of the largest principal angle between two
  column spans, checked on subspaces built at known angles (so a Frobenius norm
  in place of the 2-norm, or a missing orthonormalisation of the inputs, fails).
* ``gershgorin``: the Gershgorin interval of the Hermitian band (centre Re b_ii,
  radius sum_{j != i} |b_ij| over the whole row, i.e. both the stored lower part
  and its conjugate upper part), checked against closed forms and containment of
  the spectrum.
* ``orth`` / ``orth_max``: ||X^H X - I||_max / n (the paper's Orth, Section 4)
  and the same without the 1/n, on bases whose departure is known exactly.
"""
import numpy as np
import pytest

import oracle
import synth


def _orthonormal_pair(n, k, seed, cplx):
    g = np.random.default_rng(seed)
    Z = g.normal(size=(n, 2 * k)) + (1j * g.normal(size=(n, 2 * k)) if cplx else 0)
    Q, _ = np.linalg.qr(Z)
    return Q[:, :k], Q[:, k:]


@pytest.mark.parametrize("cplx", [False, True])
def test_sin_angle_of_subspaces_at_known_angles(cplx):
    n, k = 40, 3
    U, W = _orthonormal_pair(n, k, 7, cplx)
    theta = np.array([0.3, 0.1, 1.2])
    Xb = U * np.cos(theta)[None, :] + W * np.sin(theta)[None, :]
    assert abs(oracle.subspace_sin_angle(U, Xb) - np.sin(1.2)) <= 1e-14
    assert abs(oracle.subspace_sin_angle(Xb, U) - np.sin(1.2)) <= 1e-14
    # a Frobenius norm would report sqrt(sum sin^2) instead
    assert np.sqrt(np.sum(np.sin(theta) ** 2)) - np.sin(1.2) > 0.05
    # the spans, not the bases, decide: well-conditioned changes of basis leave the angle
    g = np.random.default_rng(3)
    Ra = np.eye(k) + 0.5 * g.normal(size=(k, k))
    Rb = np.diag([1e3, 1.0, 1e-3]) @ (np.eye(k) + 0.3 * g.normal(size=(k, k)))
    # (Rb has condition ~1e6, so the QR inside loses ~1e6 ulps)
    assert abs(oracle.subspace_sin_angle(U @ Ra, Xb @ Rb) - np.sin(1.2)) <= 1e-10
    # same span, orthogonal spans
    assert oracle.subspace_sin_angle(U, U @ Ra) <= 1e-14
    assert abs(oracle.subspace_sin_angle(U, W) - 1.0) <= 1e-14
    # columnwise phases (complex) or signs do not change a span
    ph = np.exp(1j * np.array([0.4, 2.0, -1.0])) if cplx else np.array([-1.0, 1.0, -1.0])
    assert abs(oracle.subspace_sin_angle(U * ph[None, :], Xb) - np.sin(1.2)) <= 1e-14


def test_sin_angle_small_angles_keep_relative_accuracy():
    # the eigenvector criterion is 1e-8: the helper must resolve angles far below that
    U, W = _orthonormal_pair(200, 5, 11, True)
    t = 3e-11
    Xb = U.copy()
    Xb[:, 2] = np.cos(t) * U[:, 2] + np.sin(t) * W[:, 0]
    s = oracle.subspace_sin_angle(U, Xb)
    assert abs(s - np.sin(t)) <= 1e-3 * t


def test_gershgorin_diagonal_band_is_its_diagonal():
    d = np.array([0.5, -1.25, 2.0, -3.5, 0.0, 3.0])
    for cplx in (False, True):
        lo, hi = oracle.gershgorin(synth.diagonal_band(d, 2, cplx))
        assert (lo, hi) == (-3.5, 3.0)


@pytest.mark.parametrize("c", [0.25, -0.5, 3 + 4j])
def test_gershgorin_toeplitz_tridiagonal_closed_form(c):
    n, a = 9, 0.75
    ab = np.zeros((n, 2), dtype=np.complex128 if isinstance(c, complex) else np.float64)
    ab[:, 0] = a
    ab[:-1, 1] = c
    lo, hi = oracle.gershgorin(ab)
    # interior rows carry two off-diagonal entries, the end rows one
    assert (lo, hi) == (a - 2 * abs(c), a + 2 * abs(c))


def test_gershgorin_counts_the_conjugate_upper_part():
    # one stored entry B(3, 1) = 3 + 4i also sits in row 1 as conj(B(3, 1)), modulus 5
    n, b = 5, 2
    ab = np.zeros((n, b + 1), dtype=np.complex128)
    ab[:, 0] = np.arange(n)
    ab[1, 2] = 3 + 4j                                 # column 1, row 1 + 2 = 3
    lo, hi = oracle.gershgorin(ab)
    assert (lo, hi) == (1 - 5.0, 3 + 5.0)


@pytest.mark.parametrize("cplx,b", [(False, 1), (True, 6), (False, 17), (True, 40)])
def test_gershgorin_contains_the_spectrum(cplx, b):
    ab = synth.random_band(150, b, 60 + b, cplx)
    ev = np.linalg.eigvalsh(synth.band_to_dense(ab))
    lo, hi = oracle.gershgorin(ab)
    A = synth.band_to_dense(ab)
    R = np.sum(np.abs(A), axis=1) - np.abs(np.diag(A))
    assert lo <= ev[0] and ev[-1] <= hi
    assert abs(lo - np.min(np.diag(A).real - R)) <= 1e-14 * max(1, abs(lo))
    assert abs(hi - np.max(np.diag(A).real + R)) <= 1e-14 * max(1, abs(hi))


def test_orth_known_departures():
    U, _ = _orthonormal_pair(64, 6, 5, True)
    assert oracle.orth_max(U) <= 1e-14
    eps = 2.0 ** -20
    X = U.copy()
    X[:, 4] *= 1 + eps                               # Gram entry (4, 4) becomes (1 + eps)^2
    dep = (1 + eps) ** 2 - 1
    assert abs(oracle.orth_max(X) - dep) <= 1e-15
    assert abs(oracle.orth(X) - dep / 64) <= 1e-17
    Y = U.copy()
    Y[:, 1] += 1e-6 * U[:, 3]                         # off-diagonal Gram entries 1e-6
    assert abs(oracle.orth_max(Y) - 1e-6) <= 1e-15


def test_random_start_stream_definition():
    """The start-vector stream: SplitMix64 words (the published generator, pinned by its
    golden outputs in test_oracle_slicer) mapped to [-1, 1) exactly; column c of a block that
    starts at column col0 is column col0 + c of the whole stream."""
    from oracle import slicer_oracle as so
    n, seed = 7, 12345
    X = oracle.random_start(n, 5, False, seed)
    for c in range(5):
        for i in range(n):
            w = so.splitmix64(seed + c * n + i)
            assert X[i, c] == (w >> 11) * 2.0 ** -52 - 1.0
    Z = oracle.random_start(n, 3, True, seed, col0=2)
    for c in range(3):
        for i in range(n):
            k = (2 + c) * n + i
            assert Z[i, c].real == (so.splitmix64(seed + 2 * k) >> 11) * 2.0 ** -52 - 1.0
            assert Z[i, c].imag == (so.splitmix64(seed + 2 * k + 1) >> 11) * 2.0 ** -52 - 1.0
    big = oracle.random_start(400, 50, True, 7)
    assert -1.0 <= big.real.min() and big.real.max() < 1.0
    assert abs(big.real.mean()) < 0.02 and abs(np.var(big.imag) - 1.0 / 3.0) < 0.02
