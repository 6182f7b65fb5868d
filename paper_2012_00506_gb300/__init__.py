"""GB300 (sm_103a) banded FEAST spectrum slicing -- Python binding.

A thin ``ctypes`` layer over ``libpdeshep.so`` (declared in
``include/pdeshep.h``): it marshals PyTorch CUDA tensors into device pointers,
sizes and the caller-owned workspace, and calls the C ABI.  Every step of the
computation runs in the library's CUDA kernels; there is no CPU fallback --
if the library or a GPU is missing, calls raise.

Layouts (see the header): a band is a tensor of shape ``(n, ldab)`` (float64
or complex128), row ``j`` holding ``B[j + d, j]`` for ``d = 0..b``; a block of
``m`` vectors of length ``n`` is a contiguous tensor of shape ``(m, n)`` (row
``c`` is vector ``c``), i.e. the column-major ``n x m`` matrix of the C ABI.
"""
from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libpdeshep.so")

FP64 = 0
MIXED = 1
RR_FLOATFLOAT = 0
RR_FP64 = 1
RR_TENSOR = 2
GEMM_AHB = 0
GEMM_GRAM = 1
GEMM_UPDATE = 2
PART_KMEANS = 0
PART_EQUAL_COUNT = 1
PART_EQUAL_WIDTH = 2
REFINE_NONE = 0
REFINE_RESIDUAL = 1

STATUS = {
    0: "ok", 1: "not converged", 2: "count mismatch", 3: "cholqr breakdown", 4: "non-finite input",
    5: "workspace too small", 6: "device timeout", 7: "singular", 8: "cuda error",
    9: "eig not converged",
}

EXPORTED = [
    "pdeshep_opts_default", "pdeshep_status_string", "pdeshep_last_error", "pdeshep_version",
    "pdeshep_kernel_launches", "pdeshep_alu_peak", "pdeshep_debug_wait_limit",
    "pdeshep_inertia_workspace_size", "pdeshep_inertia", "pdeshep_inertia_noalloc",
    "pdeshep_bisect_workspace_size",
    "pdeshep_bisect", "pdeshep_gershgorin", "pdeshep_contour_rule", "pdeshep_contour_rule_trapezoid",
    "pdeshep_contour_rule_zolotarev",
    "pdeshep_shifted_solve_workspace_size", "pdeshep_shifted_solve", "pdeshep_band_matmul",
    "pdeshep_cholqr_workspace_size", "pdeshep_cholqr", "pdeshep_eigh_workspace_size",
    "pdeshep_eigh", "pdeshep_workspace_size", "pdeshep_band_slice",
    "pdeshep_mlp_param_count", "pdeshep_slice_features_workspace_size", "pdeshep_slice_features",
    "pdeshep_mlp_workspace_size", "pdeshep_mlp_forward", "pdeshep_mlp_grad", "pdeshep_mlp_train_step",
    "pdeshep_propose_workspace_size", "pdeshep_propose_slices", "pdeshep_tune_reset",
    "pdeshep_block_gemm_workspace_size", "pdeshep_block_gemm",
    "pdeshep_band_matmul_tc_workspace_size", "pdeshep_band_matmul_tc",
    "pdeshep_partition", "pdeshep_outer_bounds_workspace_size", "pdeshep_outer_bounds",
    "pdeshep_restart_plan", "pdeshep_random_start", "pdeshep_equal_count_targets_workspace_size",
    "pdeshep_equal_count_targets", "pdeshep_gather_columns_workspace_size", "pdeshep_gather_columns",
]


class c128(C.Structure):
    _fields_ = [("re", C.c_double), ("im", C.c_double)]


class Opts(C.Structure):
    _fields_ = [
        ("tol", C.c_double), ("max_iter", C.c_int32), ("precision", C.c_int32),
        ("refine_policy", C.c_int32), ("rhs_chunk", C.c_int32), ("ellipse_ratio", C.c_double),
        ("bnorm", C.c_double), ("seed", C.c_uint64), ("hbm_cap_bytes", C.c_size_t),
        ("autotune", C.c_int32), ("verbose", C.c_int32), ("stream", C.c_void_p),
        ("rr_arith", C.c_int32), ("m0_resize", C.c_int32), ("tune_cache", C.c_char_p),
        ("graphs", C.c_int32), ("m0_cap", C.c_int32), ("h_m0_used", C.c_void_p),
    ]


KERNEL_GROUPS = ["inertia", "factor", "solve", "accum", "gemm", "small", "bandmm", "eig"]


class Stats(C.Structure):
    _fields_ = [
        ("iterations", C.c_int32), ("waves", C.c_int32), ("factorizations", C.c_int64),
        ("rhs_sweeps", C.c_int64), ("ms_inertia", C.c_double), ("ms_factor", C.c_double),
        ("ms_solve", C.c_double), ("ms_rr", C.c_double), ("ms_total", C.c_double),
        ("max_residual", C.c_double), ("min_rel_error_est", C.c_double),
        ("kg_ms", C.c_double * 8), ("kg_launches", C.c_int64 * 8), ("kg_flops", C.c_double * 8),
        ("rhs_columns", C.c_int64), ("cluster_ctas", C.c_int32), ("jacobi_sweeps64", C.c_int32),
        ("jacobi_sweeps32", C.c_int32), ("rr_calls", C.c_int32),
        ("eig_refine_steps", C.c_int32), ("eig_clusters", C.c_int32), ("eig_max_cluster", C.c_int32),
        ("eig_fallback_unconverged", C.c_int32), ("eig_fallback_wide", C.c_int32),
        ("rhs_chunk_used", C.c_int32), ("gram_splits_used", C.c_int32), ("tuned", C.c_int32),
        ("graph_launches", C.c_int32), ("cholqr_shifted", C.c_int32), ("gram_fp64", C.c_int32),
        ("rr_fp64_from", C.c_int32), ("rhs_chunk_early", C.c_int32),
    ]

    def as_dict(self):
        out = {}
        for k, _ in self._fields_:
            v = getattr(self, k)
            if k.startswith("kg_"):
                v = {g: float(v[i]) if k != "kg_launches" else int(v[i]) for i, g in enumerate(KERNEL_GROUPS)}
            out[k] = v
        return out


class PdeshepError(RuntimeError):
    def __init__(self, fn, status, msg=""):
        self.status = status
        text = STATUS.get(status, "invalid argument %d" % -status if status < 0 else str(status))
        super().__init__(f"{fn} failed: {text}" + (f" ({msg})" if msg else ""))


_lib = None


def load(path: str = LIB_PATH):
    """Load ``libpdeshep.so`` (build it first with ``build.build()``)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"{path} is missing: run paper_2012_00506_gb300/build.py (nvcc, sm_103a)")
    lib = C.CDLL(path)
    P, i64, i32, dbl, sz = C.c_void_p, C.c_int64, C.c_int32, C.c_double, C.c_size_t
    sig = {
        "pdeshep_opts_default": (None, [C.POINTER(Opts)]),
        "pdeshep_status_string": (C.c_char_p, [C.c_int]),
        "pdeshep_last_error": (C.c_char_p, []),
        "pdeshep_version": (C.c_char_p, []),
        "pdeshep_kernel_launches": (C.c_uint64, []),
        "pdeshep_inertia_workspace_size": (sz, [i64, i32, i32, i32]),
        "pdeshep_inertia": (C.c_int, [i64, i32, i32, P, i64, i32, P, P, P, P, sz, P]),
        "pdeshep_inertia_noalloc": (C.c_int, [i64, i32, i32, P, i64, i32, P, P, P]),
        "pdeshep_bisect_workspace_size": (sz, [i64, i32, i32, i32, i32]),
        "pdeshep_bisect": (C.c_int, [i64, i32, i32, P, i64, i32, P, dbl, i32, P, P, P, sz, P]),
        "pdeshep_gershgorin": (C.c_int, [i64, i32, i32, P, i64, P, P, P, sz, P]),
        "pdeshep_contour_rule": (C.c_int, [i32, dbl, dbl, dbl, P, P]),
        "pdeshep_contour_rule_trapezoid": (C.c_int, [i32, dbl, dbl, dbl, P, P]),
        "pdeshep_contour_rule_zolotarev": (C.c_int, [i32, dbl, dbl, dbl, P, P, P]),
        "pdeshep_shifted_solve_workspace_size": (sz, [i64, i32, i32, i32, i32]),
        "pdeshep_shifted_solve": (C.c_int, [i64, i32, i32, P, i64, i32, P, i32, P, i32, i32, P, P, P, sz, P]),
        "pdeshep_band_matmul": (C.c_int, [i64, i32, i32, P, i64, i32, P, P, P]),
        "pdeshep_cholqr_workspace_size": (sz, [i64, i32, P, i32]),
        "pdeshep_cholqr": (C.c_int, [i64, i32, i32, P, P, i32, P, P, sz, P]),
        "pdeshep_eigh_workspace_size": (sz, [i32, P, i32]),
        "pdeshep_block_gemm_workspace_size": (sz, [i64, i32, i32, P]),
        "pdeshep_block_gemm": (C.c_int, [i32, i32, i64, i32, i32, P, P, P, P, P, sz, P]),
        "pdeshep_band_matmul_tc_workspace_size": (sz, [i64, i32, i32, i32]),
        "pdeshep_band_matmul_tc": (C.c_int, [i64, i32, i32, P, i64, i32, P, P, P, sz, P]),
        "pdeshep_partition": (C.c_int, [i32, i64, P, i32, dbl, dbl, i32, P, P, P, P]),
        "pdeshep_restart_plan": (C.c_int, [i64, P, i32, P, P, i32, P]),
        "pdeshep_random_start": (C.c_int, [i64, i32, i64, i32, C.c_uint64, P, P]),
        "pdeshep_debug_wait_limit": (C.c_int, [i64]),
        "pdeshep_alu_peak": (C.c_int, [i32, i64, P, P, P]),
        "pdeshep_gather_columns_workspace_size": (sz, [i32]),
        "pdeshep_gather_columns": (C.c_int, [i64, i32, P, i64, i32, P, C.c_uint64, i64, P, P, sz, P]),
        "pdeshep_equal_count_targets_workspace_size": (sz, [i64, i32, i32, i32, i32]),
        "pdeshep_equal_count_targets": (C.c_int, [i64, i32, i32, P, i64, i32, dbl, i32, P, P, sz, P]),
        "pdeshep_outer_bounds_workspace_size": (sz, [i64, i32, i32]),
        "pdeshep_outer_bounds": (C.c_int, [i64, i32, i32, P, i64, i64, P, i64, i64, dbl, dbl, i32, P, P, P, P, sz,
                                           P]),
        "pdeshep_eigh": (C.c_int, [i32, i32, P, P, P, P, P, sz, P]),
        "pdeshep_workspace_size": (sz, [i64, i32, i32, i32, P, i32, C.POINTER(Opts)]),
        "pdeshep_band_slice": (C.c_int, [i64, i32, i32, P, i64, i32, P, i32, P, P, P, P, P, sz,
                                         C.POINTER(Opts), P, P, P, P, C.POINTER(Stats)]),
        "pdeshep_mlp_param_count": (i64, []),
        "pdeshep_slice_features_workspace_size": (sz, [i64, i32]),
        "pdeshep_slice_features": (C.c_int, [i64, i32, i32, P, i64, C.c_uint64, P, P, sz, P]),
        "pdeshep_mlp_workspace_size": (sz, [i32]),
        "pdeshep_mlp_forward": (C.c_int, [P, i32, P, P, P, sz, P]),
        "pdeshep_mlp_grad": (C.c_int, [P, i32, P, P, P, P, P, sz, P]),
        "pdeshep_mlp_train_step": (C.c_int, [P, P, P, i32, C.c_float, i32, P, P, P, P, sz, P]),
        "pdeshep_propose_workspace_size": (sz, [i64, i32, i32, i32, i32]),
        "pdeshep_tune_reset": (None, []),
        "pdeshep_propose_slices": (C.c_int, [i64, i32, i32, P, i64, P, C.c_uint64, dbl, dbl, i32, i32, i32,
                                             P, P, P, P, P, P, sz, P]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


def _torch():
    import torch
    return torch


def _stream(stream=None):
    torch = _torch()
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


def _ptr(t):
    return C.c_void_p(t.data_ptr()) if t is not None else C.c_void_p(0)


def _np_ptr(a):
    return a.ctypes.data_as(C.c_void_p)


def _check(fn, st):
    if st != 0:
        msg = load().pdeshep_last_error().decode() if st == 8 else ""
        raise PdeshepError(fn, st, msg)


def _workspace(nbytes, device):
    torch = _torch()
    return torch.empty(max(int(nbytes), 256), dtype=torch.uint8, device=device)


def _band_args(band, b):
    n, ldab = band.shape
    b = ldab - 1 if b is None else int(b)
    assert band.is_cuda and band.is_contiguous(), "band must be a contiguous CUDA tensor (n, ldab)"
    cplx = 1 if band.is_complex() else 0
    return n, b, cplx, ldab


# ---------------------------------------------------------------------------- entry points
def version() -> str:
    return load().pdeshep_version().decode()


def kernel_launches() -> int:
    """CUDA kernels launched by the library so far in this process."""
    return int(load().pdeshep_kernel_launches())


def inertia(band, sigmas, b=None, pivots=False, stream=None):
    """Eigenvalue counts below each sigma (pivot-free LDL^T inertia, FP64)."""
    torch = _torch()
    lib = load()
    n, b, cplx, ldab = _band_args(band, b)
    sig = np.ascontiguousarray(np.atleast_1d(np.asarray(sigmas, dtype=np.float64)))
    neg = np.zeros(sig.size, dtype=np.int64)
    ws = _workspace(lib.pdeshep_inertia_workspace_size(n, b, cplx, sig.size), band.device)
    piv = torch.empty((sig.size, n), dtype=torch.float64, device=band.device) if pivots else None
    st = lib.pdeshep_inertia(n, b, cplx, _ptr(band), ldab, sig.size, _np_ptr(sig), _np_ptr(neg), _ptr(piv),
                             _ptr(ws), ws.numel(), _stream(stream))
    _check("pdeshep_inertia", st)
    return (neg, piv) if pivots else neg


def inertia_noalloc(band, sigmas, b=None, stream=None):
    """Eigenvalue counts below each sigma without any device allocation.

    For callers that cannot give the library device memory: the scratch is a
    fixed array inside the library (limits: at most 1024 shifts; real b <= 194,
    complex b <= 149).  Calls that may overlap on the GPU share that array and
    must be serialised by the caller.
    """
    lib = load()
    n, b, cplx, ldab = _band_args(band, b)
    sig = np.ascontiguousarray(np.atleast_1d(np.asarray(sigmas, dtype=np.float64)))
    neg = np.zeros(sig.size, dtype=np.int64)
    st = lib.pdeshep_inertia_noalloc(n, b, cplx, _ptr(band), ldab, sig.size, _np_ptr(sig), _np_ptr(neg),
                                     _stream(stream))
    _check("pdeshep_inertia_noalloc", st)
    return neg


def bisect(band, idx, rtol=1e-12, fanout=8, b=None, stream=None):
    """Enclosures [lo, hi) of the eigenvalues with the given 0-based indices."""
    lib = load()
    n, b, cplx, ldab = _band_args(band, b)
    idx = np.ascontiguousarray(np.atleast_1d(np.asarray(idx, dtype=np.int64)))
    lo = np.zeros(idx.size)
    hi = np.zeros(idx.size)
    ws = _workspace(lib.pdeshep_bisect_workspace_size(n, b, cplx, idx.size, fanout), band.device)
    st = lib.pdeshep_bisect(n, b, cplx, _ptr(band), ldab, idx.size, _np_ptr(idx), float(rtol), int(fanout),
                            _np_ptr(lo), _np_ptr(hi), _ptr(ws), ws.numel(), _stream(stream))
    _check("pdeshep_bisect", st)
    return lo, hi


def gershgorin(band, b=None, stream=None):
    lib = load()
    n, b, cplx, ldab = _band_args(band, b)
    lo, hi = C.c_double(), C.c_double()
    ws = _workspace(4096, band.device)
    st = lib.pdeshep_gershgorin(n, b, cplx, _ptr(band), ldab, C.byref(lo), C.byref(hi), _ptr(ws), ws.numel(),
                                _stream(stream))
    _check("pdeshep_gershgorin", st)
    return lo.value, hi.value


def contour_rule(ne, lo, hi, rho=0.3, kind="gauss"):
    """Nodes/weights on the upper half ellipse (host computation): Gauss-Legendre
    (``kind="gauss"``, the default rule of ``band_slice``) or the midpoint trapezoid rule
    (``kind="trapezoid"``; pass it to ``band_slice`` as ``nodes`` / ``weights``)."""
    lib = load()
    z = np.zeros(ne, dtype=np.complex128)
    w = np.zeros(ne, dtype=np.complex128)
    fn = {"gauss": "pdeshep_contour_rule", "trapezoid": "pdeshep_contour_rule_trapezoid"}[kind]
    _check(fn, getattr(lib, fn)(int(ne), float(lo), float(hi), float(rho), _np_ptr(z), _np_ptr(w)))
    return z, w


def zolotarev_rule(ne, lo, hi, gap):
    """Zolotarev rule for [lo, hi] (host computation, ``gap >= 1e-8``): nodes, weights and the
    bound E on |filter - indicator| at every real x at least ``gap * (hi - lo)`` from both ends
    (plus a rounding floor: 1e-12 for gap >= 1e-4, 1e-9 at the smallest gap); pass the rule to
    ``band_slice`` as ``nodes`` / ``weights``."""
    lib = load()
    z = np.zeros(ne, dtype=np.complex128)
    w = np.zeros(ne, dtype=np.complex128)
    err = C.c_double()
    _check("pdeshep_contour_rule_zolotarev",
           lib.pdeshep_contour_rule_zolotarev(int(ne), float(lo), float(hi), float(gap), _np_ptr(z), _np_ptr(w),
                                              C.byref(err)))
    return z, w, err.value


def shifted_solve(band, shifts, rhs, trans=0, precision=FP64, b=None, return_ipiv=False, stream=None):
    """X_s = (z_s I - B)^{-1} Y (trans=0) or (z_s I - B)^{-H} Y (trans=1).

    ``rhs``: complex128 tensor (nrhs, n).  Returns complex128 tensor (nshift, nrhs, n).
    """
    torch = _torch()
    lib = load()
    n, b, cplx, ldab = _band_args(band, b)
    sh = np.ascontiguousarray(np.atleast_1d(np.asarray(shifts, dtype=np.complex128)))
    rhs = rhs.to(torch.complex128).contiguous()
    nrhs = rhs.shape[0]
    assert rhs.shape[1] == n
    x = torch.empty((sh.size, nrhs, n), dtype=torch.complex128, device=band.device)
    ipiv = torch.empty((sh.size, n), dtype=torch.int32, device=band.device) if return_ipiv else None
    ws = _workspace(lib.pdeshep_shifted_solve_workspace_size(n, b, sh.size, nrhs, precision), band.device)
    st = lib.pdeshep_shifted_solve(n, b, cplx, _ptr(band), ldab, sh.size, _np_ptr(sh), nrhs, _ptr(rhs),
                                   int(trans), int(precision), _ptr(x), _ptr(ipiv), _ptr(ws), ws.numel(),
                                   _stream(stream))
    _check("pdeshep_shifted_solve", st)
    return (x, ipiv) if return_ipiv else x


def band_matmul(band, X, b=None, stream=None):
    """Y = B X; X of shape (m, n) (float64 for real B, complex128 for complex B)."""
    torch = _torch()
    lib = load()
    n, b, cplx, ldab = _band_args(band, b)
    X = X.to(band.dtype).contiguous()
    Y = torch.empty_like(X)
    st = lib.pdeshep_band_matmul(n, b, cplx, _ptr(band), ldab, X.shape[0], _ptr(X), _ptr(Y), _stream(stream))
    _check("pdeshep_band_matmul", st)
    return Y


def cholqr(Q, sizes, passes=2, stream=None):
    """CholQR on column blocks of Q (shape (sum(sizes), n)); returns (Q_orth, [R_t])."""
    torch = _torch()
    lib = load()
    Q = Q.clone().contiguous()
    n = Q.shape[1]
    cplx = 1 if Q.is_complex() else 0
    m = np.ascontiguousarray(np.asarray(sizes, dtype=np.int32))
    R = torch.empty(int(np.sum(m.astype(np.int64) ** 2)), dtype=Q.dtype, device=Q.device)
    ws = _workspace(lib.pdeshep_cholqr_workspace_size(n, m.size, _np_ptr(m), cplx), Q.device)
    st = lib.pdeshep_cholqr(n, cplx, m.size, _np_ptr(m), _ptr(Q), int(passes), _ptr(R), _ptr(ws), ws.numel(),
                            _stream(stream))
    _check("pdeshep_cholqr", st)
    out, off = [], 0
    for mt in m:
        out.append(R[off: off + mt * mt].reshape(mt, mt).T)  # column-major -> (row, col)
        off += mt * mt
    return Q, out


def partition(evals, K, b0, bK, method=PART_KMEANS, max_sweeps=1000):
    """Slices for the next matrix of a sequence from the previous eigenvalues (host only):
    returns (bounds, counts, sweeps); see ``pdeshep_partition``."""
    lib = load()
    d = np.ascontiguousarray(np.sort(np.asarray(evals, dtype=np.float64)))
    bounds = np.zeros(int(K) + 1)
    counts = np.zeros(int(K), dtype=np.int32)
    kout = C.c_int32()
    sweeps = C.c_int32()
    st = lib.pdeshep_partition(int(method), d.size, _np_ptr(d), int(K), float(b0), float(bK), int(max_sweeps),
                               _np_ptr(bounds), _np_ptr(counts), C.byref(kout), C.byref(sweeps))
    _check("pdeshep_partition", st)
    k = kout.value
    return bounds[: k + 1].copy(), counts[:k].copy(), int(sweeps.value)


def restart_plan(prev_vals, bounds, m0, mode=0):
    """Previous columns (or -1 = random) for the start block of every new slice (host only);
    returns one array per slice.  See ``pdeshep_restart_plan``."""
    lib = load()
    v = np.ascontiguousarray(np.asarray(prev_vals, dtype=np.float64))
    bd = np.ascontiguousarray(np.asarray(bounds, dtype=np.float64))
    m = np.ascontiguousarray(np.asarray(m0, dtype=np.int32))
    src = np.zeros(int(m.astype(np.int64).sum()), dtype=np.int64)
    st = lib.pdeshep_restart_plan(v.size, _np_ptr(v), m.size, _np_ptr(bd), _np_ptr(m), int(mode), _np_ptr(src))
    _check("pdeshep_restart_plan", st)
    return np.split(src, np.cumsum(m)[:-1])


def gather_columns(prev, src, n=None, seed=0, col0=0, stream=None):
    """The start block (ncols, n) of a re-sliced call: row j is row src[j] of ``prev`` (a (nprev, n)
    tensor of previous eigenvectors) or, for src[j] < 0, column col0 + j of the library's start-vector
    stream (the device side of ``restart_plan``)."""
    torch = _torch()
    lib = load()
    src = np.ascontiguousarray(np.asarray(src, dtype=np.int64).reshape(-1))
    nprev, nn = prev.shape
    out = torch.empty((src.size, nn), dtype=prev.dtype, device=prev.device)
    ws = _workspace(lib.pdeshep_gather_columns_workspace_size(src.size), prev.device)
    st = lib.pdeshep_gather_columns(nn, int(prev.is_complex()), _ptr(prev), nprev, src.size, _np_ptr(src),
                                    C.c_uint64(seed), int(col0), _ptr(out), _ptr(ws), ws.numel(), _stream(stream))
    _check("pdeshep_gather_columns", st)
    return out


def outer_bounds(band, prev, i0, nev, alpha=1e-3, m_hat=6.0, max_it=64, b=None, stream=None):
    """(b0, bK, (counts taken for b0, for bK), ok) enclosing the wanted eigenvalues
    i0..i0+nev-1 of the band, searched from the previous eigenvalues ``prev`` (Algorithm 4);
    ok is False when a search stopped at max_it short of its target (PDESHEP_NOT_CONVERGED)."""
    lib = load()
    n, b, cplx, ldab = _band_args(band, b)
    d = np.ascontiguousarray(np.sort(np.asarray(prev, dtype=np.float64)))
    b0 = C.c_double()
    bK = C.c_double()
    iters = np.zeros(2, dtype=np.int32)
    ws = _workspace(lib.pdeshep_outer_bounds_workspace_size(n, b, cplx), band.device)
    st = lib.pdeshep_outer_bounds(n, b, cplx, _ptr(band), ldab, d.size, _np_ptr(d), int(i0), int(nev), float(alpha),
                                  float(m_hat), int(max_it), C.byref(b0), C.byref(bK), _np_ptr(iters), _ptr(ws),
                                  ws.numel(), _stream(stream))
    if st != 1:
        _check("pdeshep_outer_bounds", st)
    return b0.value, bK.value, (int(iters[0]), int(iters[1])), st == 0


def band_matmul_tc(band, X, b=None, stream=None):
    """Y = B X (X of shape (ncols, n), i.e. column-major n x ncols) on the tensor cores."""
    torch = _torch()
    lib = load()
    n, b, cplx, ldab = _band_args(band, b)
    X = X.to(band.dtype).contiguous()
    Y = torch.empty_like(X)
    ws = _workspace(lib.pdeshep_band_matmul_tc_workspace_size(n, b, cplx, X.shape[0]), band.device)
    st = lib.pdeshep_band_matmul_tc(n, b, cplx, _ptr(band), ldab, X.shape[0], _ptr(X), _ptr(Y), _ptr(ws),
                                    ws.numel(), _stream(stream))
    _check("pdeshep_band_matmul_tc", st)
    return Y


def block_gemm(kind, A, sizes, B=None, arith=RR_TENSOR, stream=None):
    """Batched tall products of the Rayleigh-Ritz step on column blocks.

    ``A`` (and ``B`` for GEMM_AHB): tensors of shape (sum(sizes), n), i.e. column-major
    n x sum(sizes), block t holding sizes[t] columns.  GEMM_AHB / GEMM_GRAM return the list
    [A_t^H B_t] (B_t = A_t for the Gram matrix) of (m_t, m_t) tensors; GEMM_UPDATE takes
    ``B`` as a list of (m_t, m_t) tensors and returns the blocks A_t B_t in the layout of A.
    ``arith``: RR_TENSOR (tensor-core digit products), RR_FLOATFLOAT or RR_FP64."""
    torch = _torch()
    lib = load()
    A = A.contiguous()
    n = A.shape[1]
    cplx = 1 if A.is_complex() else 0
    m = np.ascontiguousarray(np.asarray(sizes, dtype=np.int32))
    msq = int(np.sum(m.astype(np.int64) ** 2))
    if kind == GEMM_UPDATE:
        Bd = torch.cat([b_.to(A.dtype).T.contiguous().reshape(-1) for b_ in B])
        Cm = torch.empty_like(A)
    else:
        Bd = A if kind == GEMM_GRAM else B.to(A.dtype).contiguous()
        Cm = torch.empty(msq, dtype=A.dtype, device=A.device)
    ws = _workspace(lib.pdeshep_block_gemm_workspace_size(n, cplx, m.size, _np_ptr(m)), A.device)
    st = lib.pdeshep_block_gemm(int(kind), int(arith), n, cplx, m.size, _np_ptr(m), _ptr(A), _ptr(Bd), _ptr(Cm),
                                _ptr(ws), ws.numel(), _stream(stream))
    _check("pdeshep_block_gemm", st)
    if kind == GEMM_UPDATE:
        return Cm
    out, off = [], 0
    for mt in m:
        out.append(Cm[off: off + mt * mt].reshape(mt, mt).T)
        off += mt * mt
    return out


def eigh(blocks, stream=None):
    """Batched Hermitian eigensolver: list of (m, m) tensors -> list of (lam, V) (V[:, k] eigenvector)."""
    torch = _torch()
    lib = load()
    dt = blocks[0].dtype
    cplx = 1 if blocks[0].is_complex() else 0
    m = np.asarray([b_.shape[0] for b_ in blocks], dtype=np.int32)
    A = torch.cat([b_.to(dt).T.contiguous().reshape(-1) for b_ in blocks])  # column-major blocks
    lam = torch.empty(int(m.sum()), dtype=torch.float64, device=A.device)
    V = torch.empty_like(A)
    ws = _workspace(lib.pdeshep_eigh_workspace_size(m.size, _np_ptr(m), cplx), A.device)
    st = lib.pdeshep_eigh(cplx, m.size, _np_ptr(m), _ptr(A), _ptr(lam), _ptr(V), _ptr(ws), ws.numel(),
                          _stream(stream))
    _check("pdeshep_eigh", st)
    out, off, voff = [], 0, 0
    for mt in m:
        out.append((lam[voff: voff + mt], V[off: off + mt * mt].reshape(mt, mt).T))
        off += mt * mt
        voff += mt
    return out


def default_opts(**kw) -> Opts:
    o = Opts()
    load().pdeshep_opts_default(C.byref(o))
    for k, v in kw.items():
        if k == "tune_cache" and isinstance(v, str):
            v = v.encode()
        setattr(o, k, v)
    return o


def workspace_size(n, b, is_complex, m0, ne=8, opts=None) -> int:
    lib = load()
    o = opts if opts is not None else default_opts()
    m = np.ascontiguousarray(np.asarray(m0, dtype=np.int32))
    return int(lib.pdeshep_workspace_size(n, b, int(is_complex), m.size, _np_ptr(m), ne, C.byref(o)))


@dataclass
class SliceResult:
    status: int
    evals: object
    evecs: object
    counts: np.ndarray
    nfound: np.ndarray
    stats: dict = field(default_factory=dict)
    m0: np.ndarray = None
    block: int = 0        # columns per slice block (m0_resize mode); 0: blocks of m0[i] columns

    def offset(self, i):
        """First row of slice i's block in evals / evecs."""
        return i * self.block if self.block else int(np.sum(self.m0[:i]))

    def slice_pairs(self, i):
        """(eigenvalues, eigenvectors (k, n)) of the converged pairs of slice i."""
        off = self.offset(i)
        k = int(self.nfound[i])
        return self.evals[off: off + k], self.evecs[off: off + k]


def alu_peak(fp64, iters=4096, device=None, stream=None):
    """Measured FP32 (fp64=False) or FP64 FMA throughput of the GPU in TFLOP/s."""
    torch = _torch()
    lib = load()
    scratch = torch.empty(1 << 22, dtype=torch.float64, device=device)
    out = C.c_double()
    st = lib.pdeshep_alu_peak(int(bool(fp64)), int(iters), C.byref(out), _ptr(scratch), _stream(stream))
    _check("pdeshep_alu_peak", st)
    return out.value


def random_start(n, ncols, is_complex, seed=0, col0=0, device=None, stream=None):
    """Columns col0 .. col0+ncols-1 of the library's start-vector stream, as a tensor (ncols, n)
    (the vectors pdeshep_band_slice draws when it is given no start vectors)."""
    torch = _torch()
    lib = load()
    dt = torch.complex128 if is_complex else torch.float64
    x = torch.empty((ncols, n), dtype=dt, device=device)
    st = lib.pdeshep_random_start(int(n), int(bool(is_complex)), int(col0), int(ncols), C.c_uint64(seed), _ptr(x),
                                  _stream(stream))
    _check("pdeshep_random_start", st)
    return x


def band_slice(band, bounds, m0, x0, ne=8, nodes=None, weights=None, workspace=None, stream=None,
               b=None, raise_on_error=True, **opts) -> SliceResult:
    """FEAST on every slice [bounds[i], bounds[i+1]) (Algorithm 1 per slice).

    ``x0``: start vectors, tensor (sum(m0), n) of the band's dtype, or None (drawn by the
    library from ``seed``).  With ``m0_resize=1`` and ``m0_cap``: blocks of ``m0_cap`` columns
    per slice (x0 of shape (K * m0_cap, n)), m0 enlarged by the library where the exact count
    asks for it; the m0 used is in ``result.m0``.  Options: any ``Opts`` field (tol, max_iter,
    precision, refine_policy, ellipse_ratio, bnorm, hbm_cap_bytes, seed, ...).
    """
    torch = _torch()
    lib = load()
    n, b, cplx, ldab = _band_args(band, b)
    bnd = np.ascontiguousarray(np.asarray(bounds, dtype=np.float64))
    K = bnd.size - 1
    m = np.ascontiguousarray(np.asarray(m0, dtype=np.int32))
    assert m.size == K
    o = default_opts(**opts)
    o.stream = _stream(stream).value
    m_used = np.zeros(K, dtype=np.int32)
    o.h_m0_used = m_used.ctypes.data
    ncol = K * int(o.m0_cap) if o.m0_resize else int(m.sum())
    if x0 is not None:
        x0 = x0.to(band.dtype).contiguous()
        assert x0.shape == (ncol, n)
    if nodes is not None:
        nz = np.ascontiguousarray(np.asarray(nodes, dtype=np.complex128).reshape(-1))
        nw = np.ascontiguousarray(np.asarray(weights, dtype=np.complex128).reshape(-1))
        ne = nz.size // K
    else:
        nz = nw = None
    if workspace is None:
        workspace = _workspace(lib.pdeshep_workspace_size(n, b, cplx, K, _np_ptr(m), ne, C.byref(o)), band.device)
    evals = torch.empty(ncol, dtype=torch.float64, device=band.device)
    evecs = torch.empty((ncol, n), dtype=band.dtype, device=band.device)
    counts = np.zeros(K, dtype=np.int32)
    nfound = np.zeros(K, dtype=np.int32)
    stats = Stats()
    st = lib.pdeshep_band_slice(n, b, cplx, _ptr(band), ldab, K, _np_ptr(bnd), int(ne),
                                _np_ptr(nz) if nz is not None else None,
                                _np_ptr(nw) if nw is not None else None, _np_ptr(m),
                                _ptr(x0) if x0 is not None else None,
                                _ptr(workspace), workspace.numel(), C.byref(o), _ptr(evals), _ptr(evecs),
                                _np_ptr(counts), _np_ptr(nfound), C.byref(stats))
    if st != 0 and (raise_on_error and st not in (1,)):
        _check("pdeshep_band_slice", st)
    res = SliceResult(st, evals, evecs, counts, nfound, stats.as_dict(), m_used if st >= 0 else m)
    if o.m0_resize:
        res.block = int(o.m0_cap)
    return res
