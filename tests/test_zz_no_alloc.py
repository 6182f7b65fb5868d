"""Allocation-free inertia entry point (pdeshep_inertia_noalloc).

Some callers cannot give the library any device memory: their device memory
belongs to another allocator, or they run where they may only launch work on
buffers they were handed.  For them the library offers an inertia call whose
scratch is a fixed array inside the library.  This file checks, through the C
ABI, that it returns exactly the counts of the oracle's LDL^T inertia and of
the workspace-based pdeshep_inertia on calls in a row (the array keeps the
previous call's contents, so a call must not be affected by the one before),
and that requests beyond its limits are refused.  It is collected last on
purpose.
"""
import ctypes as C

import numpy as np
import pytest

import oracle
import synth
from gpu_util import dev, to_dev

pytestmark = pytest.mark.gpu


def _noalloc(lib, band, b, sig, stream):
    n, ldab = band.shape
    cplx = 1 if band.is_complex() else 0
    sig = np.ascontiguousarray(sig, dtype=np.float64)
    neg = np.zeros(sig.size, dtype=np.int64)
    st = lib.pdeshep_inertia_noalloc(n, b, cplx, C.c_void_p(band.data_ptr()), ldab, sig.size,
                                     sig.ctypes.data_as(C.c_void_p), neg.ctypes.data_as(C.c_void_p), stream)
    return st, neg


def test_noalloc_inertia_matches_workspace_version():
    import torch
    import paper_2012_00506_gb300 as pk
    device = dev()
    lib = pk.load()
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    cases = [(synth.random_band(700, 24, 901, True), 24), (synth.random_band(513, 64, 902, False), 64),
             (synth.random_band(300, 149, 903, True), 149), (synth.random_band(400, 194, 906, False), 194)]
    for call, (ab, b) in enumerate(cases + cases[:1]):
        band = to_dev(ab, device)
        rng = np.random.default_rng(call)
        sig = np.sort(rng.uniform(-1.5, 1.5, 37 + 11 * call))
        st, neg = _noalloc(lib, band, b, sig, stream)
        assert st == 0, st
        ref = pk.inertia(band, sig)
        assert np.array_equal(neg, ref), (call, neg, ref)
        # the oracle's pivot-free LDL^T in the same operation order: identical counts
        ora = np.array([oracle.inertia(ab, s, b=b) for s in sig[:: max(1, sig.size // 9)]])
        assert np.array_equal(neg[:: max(1, sig.size // 9)], ora), (call, neg, ora)


def test_noalloc_inertia_rejects_oversized_requests():
    import torch
    import paper_2012_00506_gb300 as pk
    device = dev()
    lib = pk.load()
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    band = to_dev(synth.random_band(200, 4, 904, False), device)
    st, _ = _noalloc(lib, band, 4, np.zeros(1025), stream)
    assert st == -6 and b"1024" in lib.pdeshep_last_error()
    wide = to_dev(synth.random_band(300, 150, 905, True), device)
    st, _ = _noalloc(lib, wide, 150, np.zeros(3), stream)
    assert st == -2 and b"shared-memory" in lib.pdeshep_last_error()
    st, _ = _noalloc(lib, band, -1, np.zeros(3), stream)
    assert st == -2 and b"negative" in lib.pdeshep_last_error()
    # a refused call leaves the array usable: the next call is exact again
    st, neg = _noalloc(lib, band, 4, np.array([-0.5, 0.0, 0.5]), stream)
    ab = synth.random_band(200, 4, 904, False)
    assert st == 0 and list(neg) == [oracle.inertia(ab, s) for s in (-0.5, 0.0, 0.5)]
