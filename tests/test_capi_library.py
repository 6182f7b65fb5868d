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
