"""The give-up path of the bounded mbarrier waits in the tensor-core kernels.

A testing hook (pdeshep_debug_wait_limit) lowers the poll count of the kernels' main waits to one,
so the first wait that is not already satisfied gives up on a small problem: the call must return
PDESHEP_DEVICE_TIMEOUT (no fault, no hang: the kernels still drain, with the default limit, every
copy and product they issued), and with the default restored the same calls must succeed and match
the oracle.  No wait is left without a signal: each one is only cut short."""
import numpy as np
import pytest

import oracle
import synth
from gpu_util import block_from_dev, block_to_dev, dev, to_dev

pytestmark = pytest.mark.gpu

DEVICE_TIMEOUT = 6


@pytest.fixture(scope="module")
def device():
    return dev()


def _calls(device):
    import torch
    import paper_2012_00506_gb300 as pk
    n, b = 700, 40
    ab = synth.random_band(n, b, 91, True)
    band = to_dev(ab, device)
    X = synth.random_subspace(n, 72, 92, True)
    Xd = block_to_dev(X, device)
    shifts = np.array([0.3 + 0.1j])
    Y = synth.random_subspace(n, 130, 93, True)

    def gram():
        return pk.block_gemm(pk.GEMM_GRAM, Xd, [40, 32], arith=pk.RR_TENSOR)

    def band_product():
        return pk.band_matmul_tc(band, Xd)

    def solve():
        return pk.shifted_solve(band, shifts, block_to_dev(Y, device), trans=1, precision=pk.MIXED)
    return ab, X, Y, shifts, gram, band_product, solve


def test_wait_give_up_returns_timeout_then_recovers(device):
    import torch
    import paper_2012_00506_gb300 as pk
    lib = pk.load()
    ab, X, Y, shifts, gram, band_product, solve = _calls(device)
    assert lib.pdeshep_debug_wait_limit(1) == 0
    try:
        for fn in (gram, band_product, solve):
            with pytest.raises(pk.PdeshepError) as e:
                fn()
                torch.cuda.synchronize()
            assert e.value.status == DEVICE_TIMEOUT
    finally:
        assert lib.pdeshep_debug_wait_limit(0) == 0
    torch.cuda.synchronize()
    # the context is intact and the default limit is back: the same calls succeed
    G = [g.cpu().numpy() for g in gram()]
    off = 0
    for t, m in enumerate([40, 32]):
        Xt = X[:, off:off + m]
        nrm = np.linalg.norm(Xt, axis=0)
        assert np.max(np.abs(G[t] - Xt.conj().T @ Xt) / np.outer(nrm, nrm)) < 1e-13
        off += m
    Yb = block_from_dev(band_product())
    ref = oracle.band_matvec(ab, X)
    assert np.max(np.abs(Yb - ref)) < 1e-12 * np.max(np.abs(ref))
    Xs = block_from_dev(solve()[0])
    F, ip, _ = oracle.band_lu(ab, shifts[0])
    Xo = oracle.band_solve(F, ip, 40, Y, 1)
    assert np.max(np.abs(Xs - Xo)) / np.max(np.abs(Xo)) < 1e-4
