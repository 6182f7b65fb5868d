"""Outer bounds of the wanted eigenvalues (Section 3.2, Algorithm 4) on the GPU's inertia
counts against the oracle's search on its own inertia: identical bounds and step counts (the
host arithmetic is the same and the counts are bit-identical), and the enclosure checked
against a closed-form spectrum."""
import numpy as np
import pytest

import oracle
import synth
from gpu_util import dev, to_dev
from oracle import partition_oracle as po

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def device():
    return dev()


@pytest.mark.parametrize("i0,nev,shift", [(0, 40, 0.05), (0, 25, -0.02), (30, 50, 0.01)])
def test_outer_bounds_laplacian(device, i0, nev, shift):
    import paper_2012_00506_gb300 as pk
    m, k = 13, 11
    ab = synth.laplacian_2d_band(m, k)
    i = np.arange(1, m + 1)[:, None]
    j = np.arange(1, k + 1)[None, :]
    ev = np.sort((4 - 2 * np.cos(i * np.pi / (m + 1)) - 2 * np.cos(j * np.pi / (k + 1))).ravel())
    prev = ev - shift
    b0, bK, (it_lo, it_hi), ok = pk.outer_bounds(to_dev(ab, device), prev, i0, nev)
    ob0, obK, oit_lo, oit_hi, ook = po.outer_bounds(ab, prev, i0, nev, alpha=1e-3, m_hat=6)
    assert (b0, bK, it_lo, it_hi, ok) == (ob0, obK, oit_lo, oit_hi, ook) and ok
    assert np.sum(ev < bK) >= i0 + nev and np.sum(ev < b0) <= i0


@pytest.mark.parametrize("cplx", [False, True])
def test_outer_bounds_sequence_step(device, cplx):
    """The previous eigenvalues come from the previous matrix of an SCF-like sequence
    (B_prev = B - 1e-3 E)."""
    import paper_2012_00506_gb300 as pk
    n, b = 300, 8
    ab = synth.random_band(n, b, 91 + cplx, cplx)
    g = np.random.default_rng(92)
    E = g.standard_normal(ab.shape) + (1j * g.standard_normal(ab.shape) if cplx else 0)
    E[:, 0] = E[:, 0].real
    prev = np.linalg.eigvalsh(synth.band_to_dense(ab - 1e-3 * E))
    for i0, nev in ((0, 60), (100, 30)):
        b0, bK, its, ok = pk.outer_bounds(to_dev(ab, device), prev, i0, nev)
        ob0, obK, oit_lo, oit_hi, ook = po.outer_bounds(ab, prev, i0, nev)
        assert (b0, bK, its, ok) == (ob0, obK, (oit_lo, oit_hi), ook) and ok
        assert oracle.inertia(ab, bK) >= i0 + nev and oracle.inertia(ab, b0) <= i0


def test_outer_bounds_capped_search_reports_not_converged(device):
    """max_it too small for the upper search: the library returns PDESHEP_NOT_CONVERGED with the
    same (non-enclosing) bounds and counts as the oracle."""
    import paper_2012_00506_gb300 as pk
    m, k = 13, 11
    ab = synth.laplacian_2d_band(m, k)
    i = np.arange(1, m + 1)[:, None]
    j = np.arange(1, k + 1)[None, :]
    ev = np.sort((4 - 2 * np.cos(i * np.pi / (m + 1)) - 2 * np.cos(j * np.pi / (k + 1))).ravel())
    prev = ev - 0.05
    b0, bK, its, ok = pk.outer_bounds(to_dev(ab, device), prev, 30, 50, max_it=3)
    ob0, obK, oit_lo, oit_hi, ook = po.outer_bounds(ab, prev, 30, 50, alpha=1e-3, m_hat=6, max_it=3)
    assert (b0, bK, its, ok) == (ob0, obK, (oit_lo, oit_hi), ook)
    assert not ok and its[1] == 3


@pytest.mark.parametrize("cplx", [False, True])
def test_restart_plan_device_gather(device, cplx):
    """The device side of the restart plan: previous columns copied bit for bit, the random
    columns equal to the oracle's start-vector stream at their output column."""
    import torch
    import paper_2012_00506_gb300 as pk
    n, nprev = 300, 40
    g = np.random.default_rng(5)
    vals = np.sort(g.uniform(0, 1, nprev))
    prev = synth.random_subspace(n, nprev, 6, cplx)
    bounds = [0.0, 0.25, 0.5, 0.8, 1.0]
    m0 = [14, 9, 30, 12]
    plan = pk.restart_plan(vals, bounds, m0, mode=0)
    src = np.concatenate(plan)
    assert np.any(src < 0) and np.any(src >= 0)
    X = pk.gather_columns(torch.from_numpy(np.ascontiguousarray(prev.T)).to(device), src, seed=77, col0=11)
    got = X.cpu().numpy().T
    rnd = oracle.random_start(n, src.size, cplx, seed=77, col0=11)
    for j, sj in enumerate(src):
        ref = prev[:, sj] if sj >= 0 else rnd[:, j]
        assert np.array_equal(got[:, j], ref), j
