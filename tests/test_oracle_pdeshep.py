"""The whole of the paper's Algorithm 2 at small scale with the oracles: Step (I) dense -> band,
Step (II) FEAST spectrum slicing of the band (exact counts by inertia), Step (III) backtransform;
the eigenpairs of the dense matrix come out within the FEAST tolerance of LAPACK's."""
import numpy as np
import pytest

import oracle
from oracle import partition_oracle as po
from oracle import reduction_oracle as ro


@pytest.mark.parametrize("cplx", [False, True])
def test_pdeshep_pipeline(cplx):
    n, b, nev, K = 240, 12, 48, 4
    g = np.random.default_rng(21 + cplx)
    A = g.standard_normal((n, n)) + (1j * g.standard_normal((n, n)) if cplx else 0)
    A = 0.5 * (A + A.conj().T)
    ref = np.linalg.eigvalsh(A)
    nrm = float(np.max(np.abs(ref)))
    # Step (I)
    D, W = ro.dense_to_band(A, b)
    ab = ro.to_lower_band(D, b)
    # Step (II): slices from equal counts of the (here: reference) spectrum, counts by inertia
    spacing = float(np.median(np.diff(ref[:nev])))
    bounds, _ = po.equal_count_slices(ref[:nev], K, ref[0] - 2 * spacing, 0.5 * (ref[nev - 1] + ref[nev]))
    lams, vecs = [], []
    for i in range(len(bounds) - 1):
        cnt = oracle.inertia(ab, bounds[i + 1]) - oracle.inertia(ab, bounds[i])
        m0 = oracle.m0_rule(cnt)
        Y = g.standard_normal((n, m0)) + (1j * g.standard_normal((n, m0)) if cplx else 0)
        o = oracle.feast_slice(ab, bounds[i], bounds[i + 1], Y, ne=8, rho=0.3, tol=1e-11, bnorm=nrm,
                               max_iter=40, count=cnt)
        assert o["status"] == 0 and o["nfound"] == cnt
        lams.append(o["evals"][:cnt])
        vecs.append(o["evecs"][:, :cnt])
    lam = np.concatenate(lams)
    Xh = np.concatenate(vecs, axis=1)
    # Step (III)
    X = ro.backtransform(W, Xh)
    order = np.argsort(lam)
    assert lam.size == nev
    assert np.max(np.abs(lam[order] - ref[:nev])) <= 1e-10 * nrm
    res = np.linalg.norm(A @ X - X * lam, axis=0) / (nrm * np.linalg.norm(X, axis=0))
    assert np.max(res) <= 1e-10


@pytest.mark.parametrize("cplx", [False, True])
def test_pdeshep_pipeline_generalized(cplx):
    """The generalized problem A x = lambda B x (Section 2.1): Cholesky reduction to the standard
    problem, Steps (I)-(III) as above, x = L^{-H} x~; the lowest eigenpairs of the pencil come out
    within the FEAST tolerance of SciPy's generalized solver, B-orthonormal."""
    from scipy.linalg import eigh
    n, b, nev, K = 160, 8, 30, 3
    g = np.random.default_rng(41 + cplx)
    A = g.standard_normal((n, n)) + (1j * g.standard_normal((n, n)) if cplx else 0)
    A = 0.5 * (A + A.conj().T)
    G = g.standard_normal((n, n)) + (1j * g.standard_normal((n, n)) if cplx else 0)
    B = G @ G.conj().T / n + np.eye(n)
    ref = eigh(A, B, eigvals_only=True)
    At, L = ro.generalized_to_standard(A, B)
    nrm = float(np.max(np.abs(np.linalg.eigvalsh(At))))
    D, W = ro.dense_to_band(At, b)
    ab = ro.to_lower_band(D, b)
    spacing = float(np.median(np.diff(ref[:nev])))
    bounds, _ = po.equal_count_slices(ref[:nev], K, ref[0] - 2 * spacing, 0.5 * (ref[nev - 1] + ref[nev]))
    lams, vecs = [], []
    for i in range(len(bounds) - 1):
        cnt = oracle.inertia(ab, bounds[i + 1]) - oracle.inertia(ab, bounds[i])
        m0 = oracle.m0_rule(cnt)
        Y = g.standard_normal((n, m0)) + (1j * g.standard_normal((n, m0)) if cplx else 0)
        o = oracle.feast_slice(ab, bounds[i], bounds[i + 1], Y, ne=8, rho=0.3, tol=1e-11, bnorm=nrm,
                               max_iter=40, count=cnt)
        assert o["status"] == 0 and o["nfound"] == cnt
        lams.append(o["evals"][:cnt])
        vecs.append(o["evecs"][:, :cnt])
    lam = np.concatenate(lams)
    X = ro.standard_to_generalized(L, ro.backtransform(W, np.concatenate(vecs, axis=1)))
    order = np.argsort(lam)
    assert lam.size == nev
    assert np.max(np.abs(lam[order] - ref[:nev])) <= 1e-10 * nrm
    res = np.linalg.norm(A @ X - (B @ X) * lam, axis=0) / (nrm * np.linalg.norm(B @ X, axis=0))
    assert np.max(res) <= 1e-10
    assert np.max(np.abs(X.conj().T @ B @ X - np.eye(nev))) <= 1e-9
