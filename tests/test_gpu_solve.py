"""GPU shifted band LU + multi-RHS solves (eq. (10)) against the oracle's
gbtrf-style band LU: pivot rows identical, solutions within tolerance."""
import numpy as np
import pytest

import oracle
import synth
from gpu_util import block_from_dev, block_to_dev, dev, to_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def device():
    return dev()


CASES = [(1, 0, False, 1), (5, 2, True, 3), (70, 3, False, 2), (97, 33, True, 7), (256, 64, True, 33),
         (300, 128, False, 5), (300, 128, True, 40), (129, 31, False, 64)]


@pytest.mark.parametrize("n,b,cplx,nrhs", CASES)
@pytest.mark.parametrize("trans", [0, 1])
def test_fp64_solve_matches_oracle(device, n, b, cplx, nrhs, trans):
    import torch
    import paper_2012_00506_gb300 as pk
    ab = synth.random_band(n, b, 1000 + n + b, cplx)
    lo, hi = oracle.gershgorin(ab)
    c = 0.5 * (lo + hi)
    shifts = np.array([c + 0.05j, lo + 0.3 * (hi - lo) + 0.01j, hi - 0.1 + 0.2j])
    Y = synth.random_subspace(n, nrhs, 2000 + n, True)
    X, ipiv = pk.shifted_solve(to_dev(ab, device), shifts, block_to_dev(Y, device), trans=trans,
                               precision=pk.FP64, return_ipiv=True)
    ipiv = ipiv.cpu().numpy()
    for s, z in enumerate(shifts):
        F, ip, info = oracle.band_lu(ab, z)
        assert info == 0
        Xo = oracle.band_solve(F, ip, b, Y, trans)
        Xg = block_from_dev(X[s])
        assert np.array_equal(ipiv[s], ip)
        err = np.max(np.abs(Xg - Xo)) / np.max(np.abs(Xo))
        assert err < 1e-11, err


@pytest.mark.parametrize("n,b,cplx,nrhs", [(200, 16, True, 40), (300, 64, False, 70), (257, 128, True, 33),
                                           (1000, 128, True, 300), (130, 100, False, 5), (31, 3, True, 129)])
def test_mixed_solve_fp32_class(device, n, b, cplx, nrhs):
    import paper_2012_00506_gb300 as pk
    ab = synth.random_band(n, b, 3000 + n, cplx)
    lo, hi = oracle.gershgorin(ab)
    shifts = np.array([0.5 * (lo + hi) + 0.1j, lo + 0.2 + 0.05j])
    Y = synth.random_subspace(n, nrhs, 4000 + n, True)
    for trans in (0, 1):
        X = pk.shifted_solve(to_dev(ab, device), shifts, block_to_dev(Y, device), trans=trans, precision=pk.MIXED)
        for s, z in enumerate(shifts):
            F, ip, _ = oracle.band_lu(ab, z)
            Xo = oracle.band_solve(F, ip, b, Y, trans)
            err = np.max(np.abs(block_from_dev(X[s]) - Xo)) / np.max(np.abs(Xo))
            assert err < 1e-4, err   # complex64 with FP32 accumulation


def test_band_matmul(device):
    import paper_2012_00506_gb300 as pk
    for cplx in (False, True):
        ab = synth.random_band(333, 21, 55, cplx)
        X = synth.random_subspace(333, 9, 56, cplx)
        Y = block_from_dev(pk.band_matmul(to_dev(ab, device), block_to_dev(X, device)))
        Yo = oracle.band_matvec(ab, X)
        assert np.max(np.abs(Y - (Yo if cplx else Yo.real))) < 1e-13
