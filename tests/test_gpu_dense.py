"""GPU CholQR and small Hermitian eigensolver (Rayleigh-Ritz step of Section
2.2) against the oracle."""
import numpy as np
import pytest

import oracle
import synth
from gpu_util import block_from_dev, block_to_dev, dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def device():
    return dev()


@pytest.mark.parametrize("cplx", [False, True])
def test_cholqr_matches_oracle(device, cplx):
    import paper_2012_00506_gb300 as pk
    n = 300
    sizes = [1, 17, 64, 70]
    Q0 = synth.random_subspace(n, sum(sizes), 11, cplx)
    Q, R = pk.cholqr(block_to_dev(Q0, device), sizes, passes=1)
    Qg = block_from_dev(Q)
    off = 0
    for t, m in enumerate(sizes):
        Qo, Ro, info = oracle.cholqr(Q0[:, off:off + m])
        assert info == 0
        Rg = R[t].cpu().numpy()
        assert np.max(np.abs(Rg - Ro)) < 1e-12 * np.max(np.abs(Ro))
        assert np.max(np.abs(Qg[:, off:off + m] - Qo)) < 1e-12
        off += m
    Q2, _ = pk.cholqr(block_to_dev(Q0, device), sizes, passes=2)
    Q2 = block_from_dev(Q2)
    off = 0
    for m in sizes:
        B = Q2[:, off:off + m]
        assert np.max(np.abs(B.conj().T @ B - np.eye(m))) < 1e-14
        off += m


def test_cholqr_breakdown(device):
    import paper_2012_00506_gb300 as pk
    Q0 = np.ones((64, 3))
    with pytest.raises(pk.PdeshepError) as e:
        pk.cholqr(block_to_dev(Q0, device), [3], passes=1)
    assert e.value.status == 3


@pytest.mark.parametrize("cplx", [False, True])
def test_eigh_matches_oracle(device, cplx):
    import torch
    import paper_2012_00506_gb300 as pk
    rng = np.random.default_rng(5)
    sizes = [1, 2, 13, 64, 150]
    mats = []
    for m in sizes:
        A = rng.normal(size=(m, m)) + (1j * rng.normal(size=(m, m)) if cplx else 0)
        mats.append(0.5 * (A + A.conj().T))
    out = pk.eigh([torch.from_numpy(A).to(device) for A in mats])
    for A, (lam, V) in zip(mats, out):
        lo, Vo, sw = oracle.jacobi_eig(A)
        lam = lam.cpu().numpy()
        V = V.cpu().numpy()
        nrm = max(1.0, np.linalg.norm(A))
        assert np.max(np.abs(lam - lo)) < 1e-13 * nrm
        assert np.max(np.abs(V.conj().T @ V - np.eye(len(lam)))) < 1e-13
        assert np.linalg.norm(A @ V - V * lam) < 1e-12 * nrm
        gaps = np.min(np.abs(lo[:, None] - lo[None, :]) + np.eye(len(lo)) * 1e9, axis=1)
        for k in range(len(lo)):
            if gaps[k] > 1e-6 * nrm:
                assert np.max(np.abs(V[:, k] - Vo[:, k])) < 1e-10 * nrm / gaps[k]
