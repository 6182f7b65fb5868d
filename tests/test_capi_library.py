"""The C-ABI library builds for sm_103a, loads, and exports every symbol that
include/pdeshep.h declares.  Host-only entry points (option defaults, status
strings, the quadrature rule of Section 2.2) are exercised without a GPU."""
import ctypes as C
import os
import re

import numpy as np
import pytest

import oracle

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2012_00506_gb300 import build as b
    b.build()
    import paper_2012_00506_gb300 as pk
    return pk.load()


def _declared():
    text = open(os.path.join(ROOT, "include", "pdeshep.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(pdeshep_[a-z0-9_]+)\s*\(", text)))


def test_every_declared_symbol_is_exported(lib):
    names = _declared()
    assert len(names) >= 19
    for name in names:
        assert hasattr(lib, name), name
    import paper_2012_00506_gb300 as pk
    assert sorted(pk.EXPORTED) == names


def test_opts_defaults_and_status_strings(lib):
    import paper_2012_00506_gb300 as pk
    o = pk.default_opts()
    assert o.tol == 1e-10 and o.max_iter == 20 and o.precision == pk.MIXED
    assert o.refine_policy == pk.REFINE_RESIDUAL and o.ellipse_ratio == 0.3
    assert lib.pdeshep_status_string(0) == b"ok"
    assert lib.pdeshep_status_string(2).startswith(b"subspace")
    assert lib.pdeshep_status_string(-3) == b"invalid argument"
    assert b"sm_103a" in lib.pdeshep_version()


@pytest.mark.parametrize("ne,lo,hi,rho", [(1, -1.0, 1.0, 0.3), (8, -0.7, -0.2, 0.3), (16, 2.0, 9.0, 1.0),
                                          (12, 0.0, 1e-3, 0.5)])
def test_contour_rule_matches_oracle(lib, ne, lo, hi, rho):
    import paper_2012_00506_gb300 as pk
    z, w = pk.contour_rule(ne, lo, hi, rho)
    zo, wo = oracle.contour_rule(ne, lo, hi, rho)
    scale = max(1.0, abs(lo), abs(hi))
    assert np.max(np.abs(z - zo)) <= 4e-16 * scale * 4
    assert np.max(np.abs(w - wo)) <= 4e-16 * scale * 4


def test_argument_errors_without_gpu(lib):
    # argument validation happens before any CUDA call
    z = np.zeros(4, dtype=np.complex128)
    assert lib.pdeshep_contour_rule(0, 0.0, 1.0, 0.3, z.ctypes.data, z.ctypes.data) == -1
    assert lib.pdeshep_contour_rule(4, 1.0, 0.0, 0.3, z.ctypes.data, z.ctypes.data) == -2
    sig = np.zeros(1)
    neg = np.zeros(1, dtype=np.int64)
    assert lib.pdeshep_inertia(-1, 2, 0, None, 3, 1, sig.ctypes.data, neg.ctypes.data, None, None, 0, None) == -1
    assert lib.pdeshep_inertia(10, 2, 0, None, 3, 1, sig.ctypes.data, neg.ctypes.data, None, None, 0, None) == -4


def test_tensor_products_arguments_and_workspace(lib):
    """Host-side checks of the tensor-core entry points: the default Rayleigh-Ritz arithmetic,
    workspace sizes that grow with the problem (the digit planes of the operands and of the
    band), and argument errors returned before any CUDA call."""
    import paper_2012_00506_gb300 as pk
    assert pk.default_opts().rr_arith == pk.RR_TENSOR
    m = np.array([267, 40], dtype=np.int32)
    ws = lambda n, c: lib.pdeshep_block_gemm_workspace_size(n, c, m.size, m.ctypes.data)
    assert 0 < ws(1000, 0) < ws(1000, 1) < ws(8192, 1)
    # six bf16 digit planes of the A rows (2n elements each, rows padded per block to 128) at least
    assert ws(8192, 1) >= 6 * (256 + 128) * 2 * 8192 * 2
    wb = lambda b: lib.pdeshep_band_matmul_tc_workspace_size(8192, b, 1, 267)
    assert wb(0) < wb(64) < wb(128)
    assert wb(64) - wb(0) >= 6 * 8192 * 2 * 128 * 2   # band digits widen with the window 128 + 2b
    z = np.zeros(4)
    p = z.ctypes.data
    assert lib.pdeshep_block_gemm(3, 2, 100, 1, 2, m.ctypes.data, p, p, p, p, 1, None) == -1     # kind
    assert lib.pdeshep_block_gemm(0, 3, 100, 1, 2, m.ctypes.data, p, p, p, p, 1, None) == -2     # arith
    assert lib.pdeshep_block_gemm(0, 2, 0, 1, 2, m.ctypes.data, p, p, p, p, 1, None) == -3       # n
    assert lib.pdeshep_block_gemm(0, 2, 100, 1, 2, m.ctypes.data, p, p, p, p, 1, None) == -6     # m > n
    assert lib.pdeshep_block_gemm(0, 2, 1000, 1, 2, m.ctypes.data, p, None, p, p, 1, None) == -8  # B missing
    assert lib.pdeshep_block_gemm(1, 2, 1000, 1, 2, m.ctypes.data, p, None, None, p, 1, None) == -9
    assert lib.pdeshep_band_matmul_tc(-1, 4, 1, p, 5, 3, p, p, p, 1, None) == -1
    assert lib.pdeshep_band_matmul_tc(100, 4, 1, p, 4, 3, p, p, p, 1, None) == -5             # ldab < b + 1
    assert lib.pdeshep_band_matmul_tc(100, 4, 1, p, 5, 0, p, p, p, 1, None) == -6
