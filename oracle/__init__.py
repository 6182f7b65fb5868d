"""FP64 CPU oracle for banded FEAST spectrum slicing -- TEST INFRASTRUCTURE.

Only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` may import this package.  The CUDA
product path never does, and the two share no code: this package wraps the
plain C file ``feast_oracle.c`` (built with ``gcc -O2 -ffp-contract=off``) and
adds NumPy metric helpers.

Every function states the passage of arXiv 2012.00506 it follows:

* ``inertia``            Sylvester inertia of B - sigma I by a pivot-free
                         LDL^T / LDL^H (Section 3.2; counts per slice from the
                         inertia at both ends of the interval).
* ``gauss_legendre``,
  ``contour_rule``,
  ``filter_value``       Gauss quadrature of the Cauchy integral (Section 2.2,
                         eqs. (8)-(9)); the 1/(2 pi i) factor missing from
                         eq. (8) is included.
* ``band_lu``,
  ``band_solve``         the shifted solves (z_j I - B) Q^(j) = X of eq. (10).
* ``cholqr``             orthonormal basis of Q for the Rayleigh-Ritz step.
* ``jacobi_eig``         A_q W_q = W_q Lambda_q (Section 2.2).
* ``feast_slice``        Algorithm 1 on one slice.
* ``m0_rule``            m_i^(0) = max(1.3 m_i, m_i + 10) (Section 3.2).
* ``random_start``       the random start vectors of Algorithm 1 from a
                         counter-based SplitMix64 stream (the generator both
                         sides implement from its published definition).
* ``orth``               Orth = ||X^H X - I||_max / n (Section 4, Example 2);
                         ``orth_max`` the same without the 1/n.
* ``subspace_sin_angle`` sine of the largest principal angle between two
                         column spans (the eigenvector criterion of the tests).

Submodules (plain Python/NumPy): ``partition_oracle`` (Algorithms 3 and 4, the
restart plan), ``rules_oracle`` (the trapezoid rule), ``reduction_oracle``
(Steps (I) and (III): dense -> band reduction and backtransform),
``slicer_oracle`` (the proposer's features and network).
"""
from __future__ import annotations

import ctypes as C
import math
import os
import subprocess
import sys

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "feast_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile ``liboracle.so`` next to the source (gcc, no FMA contraction)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        cmd = ["gcc", "-O2", "-std=gnu11", "-ffp-contract=off", "-fno-fast-math", "-fPIC",
               "-shared", "-o", _LIB + ".tmp", _SRC, "-lm"]
        subprocess.check_call(cmd)
        os.replace(_LIB + ".tmp", _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is not None:
        return _lib
    build()
    lib = C.CDLL(_LIB)
    i64, i32, dbl = C.c_int64, C.c_int32, C.c_double
    P = C.c_void_p
    lib.or_pivmin_real.restype = dbl
    lib.or_pivmin_real.argtypes = [i64, i64, P, i64]
    lib.or_pivmin_complex.restype = dbl
    lib.or_pivmin_complex.argtypes = [i64, i64, P, i64]
    lib.or_inertia_real.restype = i64
    lib.or_inertia_real.argtypes = [i64, i64, P, i64, dbl, dbl, P]
    lib.or_inertia_complex.restype = i64
    lib.or_inertia_complex.argtypes = [i64, i64, P, i64, dbl, dbl, P]
    lib.or_gershgorin.restype = None
    lib.or_gershgorin.argtypes = [i64, i64, P, i64, P, P]
    lib.or_gauss_legendre.restype = None
    lib.or_gauss_legendre.argtypes = [i32, P, P]
    lib.or_contour_rule.restype = None
    lib.or_contour_rule.argtypes = [i32, dbl, dbl, dbl, P, P]
    lib.or_filter_value.restype = dbl
    lib.or_filter_value.argtypes = [i32, P, P, dbl]
    lib.or_band_lu.restype = i64
    lib.or_band_lu.argtypes = [i64, i64, P, i64, dbl, dbl, P, i64, P]
    lib.or_band_solve.restype = None
    lib.or_band_solve.argtypes = [i64, i64, P, i64, P, i32, i64, P, i64]
    lib.or_band_matvec.restype = None
    lib.or_band_matvec.argtypes = [i64, i64, P, i64, i64, P, i64, P, i64]
    lib.or_cholqr.restype = i64
    lib.or_cholqr.argtypes = [i64, i64, P, i64, P]
    lib.or_jacobi_eig.restype = i32
    lib.or_jacobi_eig.argtypes = [i64, P, P, P, dbl, i32]
    lib.or_feast_slice.restype = i32
    lib.or_feast_slice.argtypes = [i64, i64, P, i64, i32, dbl, dbl, i32, P, P, i64, P, dbl,
                                   dbl, i32, i64, P, P, P, P, P, P]
    _lib = lib
    return lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p)


def _cband(ab: np.ndarray) -> np.ndarray:
    return np.ascontiguousarray(ab, dtype=np.complex128)


def _semi(ab: np.ndarray) -> int:
    return ab.shape[1] - 1


# ----------------------------------------------------------------------------- inertia
def pivmin(ab: np.ndarray) -> float:
    """pivmin = DBL_MIN * max(1, amax^2) used in place of an exactly zero pivot."""
    lib = _load()
    n, ldab = ab.shape
    if np.iscomplexobj(ab):
        a = _cband(ab)
        return lib.or_pivmin_complex(n, ldab - 1, _ptr(a), ldab)
    a = np.ascontiguousarray(ab, dtype=np.float64)
    return lib.or_pivmin_real(n, ldab - 1, _ptr(a), ldab)


def inertia(ab: np.ndarray, sigma: float, b: int | None = None, return_pivots: bool = False):
    """Number of eigenvalues of B below ``sigma`` (negative LDL pivots of B - sigma I).

    ``b`` is the semi-bandwidth (defaults to ``ab.shape[1]-1``).  With
    ``return_pivots`` the diagonal D of the factorization is returned too.
    """
    lib = _load()
    n, ldab = ab.shape
    b = ldab - 1 if b is None else b
    d = np.zeros(n, dtype=np.float64)
    pm = pivmin(ab)
    if np.iscomplexobj(ab):
        a = _cband(ab)
        neg = lib.or_inertia_complex(n, b, _ptr(a), ldab, float(sigma), pm, _ptr(d))
    else:
        a = np.ascontiguousarray(ab, dtype=np.float64)
        neg = lib.or_inertia_real(n, b, _ptr(a), ldab, float(sigma), pm, _ptr(d))
    return (int(neg), d) if return_pivots else int(neg)


def gershgorin(ab: np.ndarray):
    """Gershgorin interval (lo, hi) containing the spectrum of B."""
    lib = _load()
    a = _cband(ab)
    n, ldab = a.shape
    lo, hi = C.c_double(), C.c_double()
    lib.or_gershgorin(n, ldab - 1, _ptr(a), ldab, C.byref(lo), C.byref(hi))
    return lo.value, hi.value


def eig_by_bisection(ab: np.ndarray, k: int, tol: float = 1e-14):
    """Enclosure [lo, hi] of the k-th smallest eigenvalue (0-based) by bisection on inertia.

    Invariant: inertia(lo) <= k < inertia(hi).  Stops when hi - lo <= tol * max(1, |hi|, |lo|).
    """
    lo, hi = gershgorin(ab)
    span = hi - lo
    lo -= 1e-3 * span + 1e-300
    hi += 1e-3 * span + 1e-300
    for _ in range(200):
        if hi - lo <= tol * max(1.0, abs(lo), abs(hi)):
            break
        mid = 0.5 * (lo + hi)
        if mid <= lo or mid >= hi:
            break
        if inertia(ab, mid) <= k:
            lo = mid
        else:
            hi = mid
    return lo, hi


def boundary_between(ab: np.ndarray, k: int, tol: float = 1e-14) -> float:
    """Slice boundary at the middle of the gap between eigenvalues k-1 and k (0-based)."""
    a = eig_by_bisection(ab, k - 1, tol)
    c = eig_by_bisection(ab, k, tol)
    sigma = 0.5 * (a[1] + c[0])
    assert inertia(ab, sigma) == k
    return sigma


def spectral_norm(ab: np.ndarray, tol: float = 1e-12) -> float:
    """||B||_2 = max(|lambda_min|, |lambda_max|) by bisection on inertia."""
    n = ab.shape[0]
    lmin = eig_by_bisection(ab, 0, tol)
    lmax = eig_by_bisection(ab, n - 1, tol)
    return max(abs(lmin[0]), abs(lmin[1]), abs(lmax[0]), abs(lmax[1]))


# ----------------------------------------------------------------------------- quadrature
def gauss_legendre(ne: int):
    """Gauss-Legendre nodes (ascending) and weights on [-1, 1]."""
    lib = _load()
    x = np.zeros(ne)
    w = np.zeros(ne)
    lib.or_gauss_legendre(ne, _ptr(x), _ptr(w))
    return x, w


def contour_rule(ne: int, lo: float, hi: float, rho: float = 0.3):
    """Upper-half ellipse nodes z_k and weights w_k for the slice [lo, hi]."""
    lib = _load()
    z = np.zeros(ne, dtype=np.complex128)
    w = np.zeros(ne, dtype=np.complex128)
    lib.or_contour_rule(ne, float(lo), float(hi), float(rho), _ptr(z), _ptr(w))
    return z, w


def filter_value(z: np.ndarray, w: np.ndarray, x: float) -> float:
    """r(x) = 2 Re sum_k w_k / (z_k - x)."""
    lib = _load()
    z = np.ascontiguousarray(z, dtype=np.complex128)
    w = np.ascontiguousarray(w, dtype=np.complex128)
    return lib.or_filter_value(len(z), _ptr(z), _ptr(w), float(x))


# ----------------------------------------------------------------------------- band LU / solves
def band_lu(ab: np.ndarray, z: complex):
    """LU with partial pivoting of z I - B: returns (F, ipiv, info), F of shape (n, 3b+1)."""
    lib = _load()
    a = _cband(ab)
    n, ldab = a.shape
    b = ldab - 1
    ldf = 3 * b + 1
    F = np.zeros((n, ldf), dtype=np.complex128)
    ipiv = np.zeros(n, dtype=np.int32)
    info = lib.or_band_lu(n, b, _ptr(a), ldab, complex(z).real, complex(z).imag, _ptr(F), ldf,
                          _ptr(ipiv))
    return F, ipiv, int(info)


def band_solve(F: np.ndarray, ipiv: np.ndarray, b: int, Y: np.ndarray, trans: int = 0):
    """Solve (zI - B) X = Y (trans=0) or (zI - B)^H X = Y (trans=1) with factors of band_lu."""
    lib = _load()
    n, ldf = F.shape
    X = np.asfortranarray(np.array(Y, dtype=np.complex128, copy=True).reshape(n, -1))
    lib.or_band_solve(n, b, _ptr(F), ldf, _ptr(np.ascontiguousarray(ipiv, dtype=np.int32)),
                      int(trans), X.shape[1], _ptr(X), n)
    return X


def band_matvec(ab: np.ndarray, X: np.ndarray) -> np.ndarray:
    """Y = B X with B the Hermitian band."""
    lib = _load()
    a = _cband(ab)
    n, ldab = a.shape
    Xc = np.asfortranarray(np.asarray(X, dtype=np.complex128).reshape(n, -1))
    Y = np.zeros_like(Xc, order="F")
    lib.or_band_matvec(n, ldab - 1, _ptr(a), ldab, Xc.shape[1], _ptr(Xc), n, _ptr(Y), n)
    return Y


# ----------------------------------------------------------------------------- small dense
def cholqr(Q: np.ndarray):
    """One CholQR pass: returns (Q R^{-1}, R, info)."""
    lib = _load()
    Qc = np.asfortranarray(np.array(Q, dtype=np.complex128, copy=True))
    n, m = Qc.shape
    R = np.zeros((m, m), dtype=np.complex128, order="F")
    info = lib.or_cholqr(n, m, _ptr(Qc), n, _ptr(R))
    return Qc, R, int(info)


def jacobi_eig(A: np.ndarray, tol: float = 1e-14, max_sweeps: int = 60):
    """Cyclic Jacobi: (eigenvalues ascending, eigenvectors, sweeps or -1)."""
    lib = _load()
    Ac = np.asfortranarray(np.array(A, dtype=np.complex128, copy=True))
    m = Ac.shape[0]
    lam = np.zeros(m)
    V = np.zeros((m, m), dtype=np.complex128, order="F")
    sw = lib.or_jacobi_eig(m, _ptr(Ac), _ptr(lam), _ptr(V), float(tol), int(max_sweeps))
    return lam, V, int(sw)


# ----------------------------------------------------------------------------- FEAST
def m0_rule(m: int) -> int:
    """Subspace size m^(0) = max(ceil(1.3 m), m + 10) (Section 3.2)."""
    return max(int(math.ceil(1.3 * m - 1e-12)), m + 10)


def feast_slice(ab: np.ndarray, lo: float, hi: float, Y0: np.ndarray, *, ne: int = 8,
                rho: float = 0.3, tol: float = 1e-10, bnorm: float | None = None,
                max_iter: int = 20, count: int | None = None, rule=None) -> dict:
    """Algorithm 1 on the slice [lo, hi) with start vectors Y0 (n x m0)."""
    lib = _load()
    a = _cband(ab)
    n, ldab = a.shape
    b = ldab - 1
    is_real = not np.iscomplexobj(ab) and not np.iscomplexobj(Y0)
    if rule is None:
        z, w = contour_rule(ne, lo, hi, rho)
    else:
        z, w = (np.ascontiguousarray(r, dtype=np.complex128) for r in rule)
        ne = len(z)
    if bnorm is None:
        bnorm = spectral_norm(ab)
    if count is None:
        count = inertia(ab, hi) - inertia(ab, lo)
    Y = np.asfortranarray(np.asarray(Y0, dtype=np.complex128))
    m0 = Y.shape[1]
    evals = np.zeros(m0)
    evecs = np.zeros((n, m0), dtype=np.complex128, order="F")
    res = np.zeros(m0)
    hist = np.zeros(max_iter)
    nfound = C.c_int64()
    iters = C.c_int32()
    st = lib.or_feast_slice(n, b, _ptr(a), ldab, int(is_real), float(lo), float(hi), ne, _ptr(z),
                            _ptr(w), m0, _ptr(Y), float(tol), float(bnorm), int(max_iter),
                            int(count), _ptr(evals), _ptr(evecs), _ptr(res), C.byref(nfound),
                            C.byref(iters), _ptr(hist))
    if is_real:
        evecs = np.asfortranarray(evecs.real)
    return dict(status=int(st), evals=evals, evecs=evecs, res=res, nfound=int(nfound.value),
                iters=int(iters.value), count=int(count), hist=hist[: int(iters.value)],
                bnorm=float(bnorm))


# ----------------------------------------------------------------------------- start vectors
def _splitmix64_array(x: np.ndarray) -> np.ndarray:
    """SplitMix64 of each uint64 state (Vigna: add 0x9e3779b97f4a7c15, then the mixer),
    arithmetic modulo 2^64."""
    z = x.astype(np.uint64) + np.uint64(0x9E3779B97F4A7C15)
    z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
    z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
    return z ^ (z >> np.uint64(31))


def random_start(n: int, ncols: int, is_complex: bool, seed: int = 0, col0: int = 0) -> np.ndarray:
    """Start vectors drawn from a counter-based stream (the "random vectors" that start
    Algorithm 1): entry (i, c) uses word k = (col0 + c) n + i; u(w) = (top 53 bits of
    splitmix64(w)) 2^-52 - 1 in [-1, 1); real: u(seed + k); complex: u(seed + 2k) + i u(seed + 2k + 1).
    Returns an n x ncols array (column-major meaning: column c is X[:, c])."""
    i = np.arange(n, dtype=np.uint64)[:, None]
    c = np.arange(ncols, dtype=np.uint64)[None, :]
    k = (np.uint64(col0) + c) * np.uint64(n) + i
    sd = np.uint64(seed & 0xFFFFFFFFFFFFFFFF)
    with np.errstate(over="ignore"):
        def u(w):
            return (_splitmix64_array(w) >> np.uint64(11)).astype(np.float64) * 2.0 ** -52 - 1.0
        if not is_complex:
            return u(sd + k)
        return u(sd + np.uint64(2) * k) + 1j * u(sd + np.uint64(2) * k + np.uint64(1))


# ----------------------------------------------------------------------------- metrics
def residuals(ab: np.ndarray, lam: np.ndarray, X: np.ndarray, bnorm: float) -> np.ndarray:
    """||B x_i - lambda_i x_i||_2 / (bnorm ||x_i||_2) per column."""
    BX = band_matvec(ab, X)
    R = BX - np.asarray(X) * lam[None, :]
    return np.linalg.norm(R, axis=0) / (bnorm * np.linalg.norm(X, axis=0))


def orth(X: np.ndarray) -> float:
    """Orth = ||X^H X - I||_max / n (Section 4, Example 2)."""
    X = np.asarray(X)
    G = X.conj().T @ X
    return float(np.max(np.abs(G - np.eye(G.shape[0]))) / X.shape[0])


def orth_max(X: np.ndarray) -> float:
    """||X^H X - I||_max without the 1/n of the paper's Orth: the largest entrywise departure
    of the Gram matrix from the identity (a validity check that does not shrink with n)."""
    X = np.asarray(X)
    G = X.conj().T @ X
    return float(np.max(np.abs(G - np.eye(G.shape[0]))))


def subspace_sin_angle(Xa: np.ndarray, Xb: np.ndarray) -> float:
    """Largest principal-angle sine between span(Xa) and span(Xb) (both full column rank)."""
    Qa, _ = np.linalg.qr(np.asarray(Xa))
    Qb, _ = np.linalg.qr(np.asarray(Xb))
    P = Qb - Qa @ (Qa.conj().T @ Qb)
    return float(np.linalg.norm(P, 2))


if __name__ == "__main__":  # pragma: no cover
    build(force="--force" in sys.argv)
    print(_LIB)
