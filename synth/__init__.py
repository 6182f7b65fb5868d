"""Seeded synthetic inputs for banded FEAST spectrum slicing.

This module is shared by the CPU oracle tests, the GPU parity tests and the
benchmark.  It only draws random numbers and lays them out; it contains none of
the eigensolver's arithmetic (no inertia, no factorization, no quadrature).

Storage convention (used everywhere in this repository)
-------------------------------------------------------
A Hermitian (or real symmetric) band matrix ``B`` of order ``n`` and
semi-bandwidth ``b`` is held in LAPACK *lower compact band* form, column-major:
entry ``B[i, j]`` for ``j <= i <= min(n-1, j+b)`` lives at ``ab[(i-j) + j*ldab]``.
In NumPy we hold it as a C-ordered array ``ab`` of shape ``(n, ldab)`` so that
``ab[j, i-j] == B[i, j]``; that is byte-for-byte the column-major layout above.
Entries that fall outside the matrix (``j + d >= n``) are zero.  The diagonal of
a complex Hermitian band has zero imaginary part.

Dense blocks of vectors (start subspaces, eigenvectors) are column-major
``n x m`` arrays, i.e. NumPy Fortran-ordered arrays of shape ``(n, m)``.

Workloads
---------
The paper's own matrices (NaCl, AuAg from FLAPW codes; Si5H12 and H2O from the
SuiteSparse collection; band reductions with semi-bandwidth 64, Section 4) are
not available here; the recipes below stand in for them:

* ``random_band``: diagonal U[-1, 1], off-diagonals N(0, s^2) (real) or
  Re, Im ~ N(0, s^2/2) (complex).
* ``mixture_band``: diagonal drawn from a mixture of Gaussians (clustered
  spectrum), off-diagonals as above.
* ``perturbation``: the random Hermitian band E_k of an SCF-like sequence
  B_{k+1} = B_k + eps * E_k (diagonal N(0,1), off-diagonals N(0,1) real or
  Re, Im ~ N(0, 1/2) complex), mirroring the slowly changing matrices of the
  SCF iterations in Section 3.
* ``laplacian_2d_band``: the 5-point Laplacian on an m-by-k grid in natural
  ordering (semi-bandwidth k); its spectrum is known in closed form.
* ``random_subspace``: the random start vectors of Algorithm 1.
"""
from __future__ import annotations

import numpy as np

__all__ = [
    "rng",
    "random_band",
    "mixture_band",
    "perturbation",
    "laplacian_2d_band",
    "diagonal_band",
    "random_subspace",
    "unitary_phases",
    "band_to_dense",
    "phase_similarity",
    "config_seed",
    "pad_band",
]


def rng(seed: int) -> np.random.Generator:
    """PCG64 generator for ``seed`` (the only RNG used for inputs)."""
    return np.random.Generator(np.random.PCG64(int(seed)))


def config_seed(config: int, replica: int = 0) -> int:
    """Seed for workload ``config`` (1-based) and ``replica``: 1000*config + replica."""
    return 1000 * int(config) + int(replica)


def _zero_outside(ab: np.ndarray) -> np.ndarray:
    n, ldab = ab.shape
    for d in range(1, ldab):
        ab[max(n - d, 0):, d] = 0
    return ab


def random_band(n: int, b: int, seed: int, is_complex: bool = False,
                off_sigma: float = 0.1, diag_lo: float = -1.0,
                diag_hi: float = 1.0) -> np.ndarray:
    """Band with diagonal U[diag_lo, diag_hi] and off-diagonal entries of std ``off_sigma``."""
    g = rng(seed)
    dtype = np.complex128 if is_complex else np.float64
    ab = np.zeros((n, b + 1), dtype=dtype)
    ab[:, 0] = g.uniform(diag_lo, diag_hi, size=n)
    if b > 0:
        if is_complex:
            s = off_sigma / np.sqrt(2.0)
            ab[:, 1:] = g.normal(0.0, s, size=(n, b)) + 1j * g.normal(0.0, s, size=(n, b))
        else:
            ab[:, 1:] = g.normal(0.0, off_sigma, size=(n, b))
    return _zero_outside(ab)


def mixture_band(n: int, b: int, seed: int, is_complex: bool = False,
                 ncomp: int = 4, comp_sigma: float = 0.05,
                 off_sigma: float = 0.02, means=None, weights=None) -> np.ndarray:
    """Band whose diagonal is drawn from a mixture of ``ncomp`` Gaussians.

    Means default to U[-1, 1] draws and weights to equal weights (clustered
    spectrum workload).  Off-diagonals have std ``off_sigma``.
    """
    g = rng(seed)
    if means is None:
        means = g.uniform(-1.0, 1.0, size=ncomp)
    means = np.asarray(means, dtype=np.float64)
    if weights is None:
        weights = np.full(len(means), 1.0 / len(means))
    weights = np.asarray(weights, dtype=np.float64)
    weights = weights / weights.sum()
    comp = g.choice(len(means), size=n, p=weights)
    dtype = np.complex128 if is_complex else np.float64
    ab = np.zeros((n, b + 1), dtype=dtype)
    ab[:, 0] = means[comp] + g.normal(0.0, comp_sigma, size=n)
    if b > 0:
        if is_complex:
            s = off_sigma / np.sqrt(2.0)
            ab[:, 1:] = g.normal(0.0, s, size=(n, b)) + 1j * g.normal(0.0, s, size=(n, b))
        else:
            ab[:, 1:] = g.normal(0.0, off_sigma, size=(n, b))
    return _zero_outside(ab)


def perturbation(n: int, b: int, seed: int, is_complex: bool) -> np.ndarray:
    """Random Hermitian band E: diagonal N(0,1), off-diagonals N(0,1) (Re, Im ~ N(0,1/2))."""
    g = rng(seed)
    dtype = np.complex128 if is_complex else np.float64
    ab = np.zeros((n, b + 1), dtype=dtype)
    ab[:, 0] = g.normal(0.0, 1.0, size=n)
    if b > 0:
        if is_complex:
            s = np.sqrt(0.5)
            ab[:, 1:] = g.normal(0.0, s, size=(n, b)) + 1j * g.normal(0.0, s, size=(n, b))
        else:
            ab[:, 1:] = g.normal(0.0, 1.0, size=(n, b))
    return _zero_outside(ab)


def laplacian_2d_band(m: int, k: int) -> np.ndarray:
    """5-point Laplacian on an m x k grid (Dirichlet), natural ordering, b = k.

    Its eigenvalues are 4 - 2cos(i*pi/(m+1)) - 2cos(j*pi/(k+1)), i=1..m, j=1..k.
    """
    n = m * k
    ab = np.zeros((n, k + 1), dtype=np.float64)
    ab[:, 0] = 4.0
    for idx in range(n):
        r, c = divmod(idx, k)
        if c + 1 < k:
            ab[idx, 1] = -1.0
        if r + 1 < m:
            ab[idx, k] = -1.0
    return ab


def diagonal_band(diag, b: int, is_complex: bool = False) -> np.ndarray:
    """Band of semi-bandwidth ``b`` holding only the given diagonal."""
    diag = np.asarray(diag, dtype=np.float64)
    ab = np.zeros((diag.size, b + 1), dtype=np.complex128 if is_complex else np.float64)
    ab[:, 0] = diag
    return ab


def random_subspace(n: int, m0: int, seed: int, is_complex: bool) -> np.ndarray:
    """Random start vectors: N(0,1) (real) or (N(0,1) + i N(0,1))/sqrt(2), column-major."""
    g = rng(seed)
    if is_complex:
        y = (g.normal(size=(m0, n)) + 1j * g.normal(size=(m0, n))) / np.sqrt(2.0)
    else:
        y = g.normal(size=(m0, n))
    return np.asfortranarray(y.T)


def unitary_phases(n: int, seed: int) -> np.ndarray:
    """Phases e^{i phi_k}, phi_k ~ U[0, 2 pi), for a unitary diagonal similarity."""
    g = rng(seed)
    return np.exp(1j * g.uniform(0.0, 2.0 * np.pi, size=n))


def phase_similarity(ab: np.ndarray, phases: np.ndarray) -> np.ndarray:
    """Band of D B D^H with D = diag(phases): entry (i, j) gets phases[i]*conj(phases[j])."""
    n, ldab = ab.shape
    out = np.zeros((n, ldab), dtype=np.complex128)
    for d in range(ldab):
        j = np.arange(n - d)
        out[j, d] = ab[j, d] * phases[j + d] * np.conj(phases[j])
    out[:, 0] = out[:, 0].real
    return out


def band_to_dense(ab: np.ndarray) -> np.ndarray:
    """Dense Hermitian matrix from the lower compact band (format conversion only)."""
    n, ldab = ab.shape
    a = np.zeros((n, n), dtype=ab.dtype)
    for d in range(ldab):
        j = np.arange(n - d)
        a[j + d, j] = ab[j, d]
        if d:
            a[j, j + d] = np.conj(ab[j, d])
    return a


def pad_band(ab: np.ndarray, ldab: int) -> np.ndarray:
    """Copy of ``ab`` with a larger leading dimension (extra rows zero)."""
    n, l0 = ab.shape
    out = np.zeros((n, ldab), dtype=ab.dtype)
    out[:, :l0] = ab
    return out
