"""The benchmark configurations at full size, in the launch configuration the bench uses.

* Config 1 (plain FP64 FEAST, real n = 2000, b = 32, one slice of eigenvalues 500-599, Ne = 8,
  m0 = 150, random start, tol 1e-10): element by element against the oracle's own FEAST run, also
  in mixed precision with float-float (arith 0) and tensor-core (arith 2) Rayleigh-Ritz products.
  Configs 2 and 3 run with both Rayleigh-Ritz arithmetics.
* Config 2 (complex n = 8192, b = 64, 8 slices over the lowest 20 %, m0 = 267, mixed
  precision): the exact counts at every boundary, the residual of every converged pair,
  orthogonality, sampled eigenvalues by bisection, and (tensor-core Rayleigh-Ritz) slice 0
  element by element against the oracle's FEAST from the same start vectors.
* Config 3 (real clustered n = 32768, b = 128, 64 slices of 40-400 eigenvalues, Ne = 16, 1024
  factorizations in slice groups under a 100 GB factor cap): the exact counts at all 65
  boundaries and the residuals of sampled slices against the oracle.
"""
import numpy as np
import pytest

import oracle
import synth
from gpu_util import block_from_dev, block_to_dev, dev, orth_tol, to_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def device():
    return dev()


@pytest.mark.parametrize("precision,arith", [(0, 0), (1, 0), (1, 2)])
def test_config1_full_size_against_oracle(device, precision, arith):
    import paper_2012_00506_gb300 as pk
    n, b = 2000, 32
    ab = synth.random_band(n, b, synth.config_seed(1), False, off_sigma=0.1)
    bounds = [oracle.boundary_between(ab, 500), oracle.boundary_between(ab, 600)]
    bnorm = oracle.spectral_norm(ab)
    X0 = synth.random_subspace(n, 150, synth.config_seed(1) + 1, False)
    r = pk.band_slice(to_dev(ab, device), bounds, [150], block_to_dev(X0, device), ne=8, precision=precision,
                      bnorm=bnorm, tol=1e-10, max_iter=40, rr_arith=arith)
    assert r.status == 0
    assert r.counts[0] == 100 == oracle.inertia(ab, bounds[1]) - oracle.inertia(ab, bounds[0])
    assert r.nfound[0] == 100
    o = oracle.feast_slice(ab, bounds[0], bounds[1], X0, ne=8, rho=0.3, tol=1e-10, bnorm=bnorm, max_iter=40,
                           count=100)
    assert o["status"] == 0 and o["nfound"] == 100
    lg = r.evals.cpu().numpy()[:100]
    Xg = block_from_dev(r.evecs)[:, :100]
    assert np.max(np.abs(lg - o["evals"][:100])) <= 1e-10 * bnorm
    assert oracle.subspace_sin_angle(Xg, o["evecs"][:, :100]) <= 1e-8
    assert np.max(oracle.residuals(ab, lg, Xg, bnorm)) <= 1e-10
    assert oracle.orth(Xg) < 1e-13
    # entrywise: FP64 products below 1e-13 here; the mixed path within n u of its products' arithmetic
    assert oracle.orth_max(Xg) <= (1e-13 if precision == 0 else orth_tol(n, arith))


@pytest.mark.parametrize("arith", [0, 2])
def test_config2_full_size_properties(device, arith):
    import paper_2012_00506_gb300 as pk
    n, b, nslice = 8192, 64, 8
    ab = synth.random_band(n, b, synth.config_seed(2), True, off_sigma=0.1)
    band = to_dev(ab, device)
    nev = int(0.2 * n)
    ks = [int(round(i * nev / nslice)) for i in range(nslice + 1)]
    idx = sorted(set(ks[1:] + [k - 1 for k in ks[1:]] + [0]))
    lo, hi = pk.bisect(band, idx, rtol=1e-12, fanout=8)
    lam = {k: 0.5 * (lo[i] + hi[i]) for i, k in enumerate(idx)}
    spacing = (lam[ks[1]] - lam[0]) / ks[1]
    bounds = [lam[0] - 2 * spacing] + [0.5 * (lam[k - 1] + lam[k]) for k in ks[1:]]
    m0 = [oracle.m0_rule(ks[i + 1] - ks[i]) for i in range(nslice)]
    bnorm = oracle.spectral_norm(ab, tol=1e-10)
    X0 = synth.random_subspace(n, int(sum(m0)), synth.config_seed(2) + 999, True)
    r = pk.band_slice(band, bounds, m0, block_to_dev(X0, device), ne=8, precision=pk.MIXED, bnorm=bnorm,
                      tol=1e-10, max_iter=40, autotune=1, rr_arith=arith)
    assert r.status == 0
    neg = [oracle.inertia(ab, s) for s in bounds]
    assert list(r.counts) == list(np.diff(neg))          # bit-exact counts at every boundary
    assert list(r.nfound) == list(r.counts)
    ev = r.evals.cpu().numpy()
    V = block_from_dev(r.evecs)
    off = 0
    found = []
    for i in range(nslice):
        k = int(r.nfound[i])
        li, Xi = ev[off:off + k], V[:, off:off + k]
        assert np.all((li >= bounds[i]) & (li < bounds[i + 1]))
        assert np.max(oracle.residuals(ab, li, Xi, bnorm)) <= 1e-10
        assert oracle.orth(Xi) < 1e-13
        assert oracle.orth_max(Xi) <= orth_tol(n, arith)
        found.append(li)
        off += m0[i]
    allev = np.sort(np.concatenate(found))
    assert allev.size == nev
    for k in (0, nev // 2, nev - 1):                      # sampled eigenvalues by bisection on inertia
        elo, ehi = oracle.eig_by_bisection(ab, k, tol=1e-13)
        assert abs(allev[k] - 0.5 * (elo + ehi)) <= 1e-10 * bnorm
    if arith == 2:                                        # a whole slice against the oracle's FEAST
        cnt = int(r.counts[0])
        o = oracle.feast_slice(ab, bounds[0], bounds[1], X0[:, :m0[0]], ne=8, rho=0.3, tol=1e-10, bnorm=bnorm,
                               max_iter=40, count=cnt)
        assert o["status"] == 0 and o["nfound"] == cnt
        assert np.max(np.abs(ev[:cnt] - o["evals"][:cnt])) <= 1e-10 * bnorm
        assert oracle.subspace_sin_angle(V[:, :cnt], o["evecs"][:, :cnt]) <= 1e-8


@pytest.mark.parametrize("arith", [0, 2])
def test_config3_uneven_slices_in_waves(device, arith):
    import paper_2012_00506_gb300 as pk
    n, b, nslice, ne = 32768, 128, 64, 16
    ab = synth.mixture_band(n, b, synth.config_seed(3), off_sigma=0.02)
    band = to_dev(ab, device)
    g = np.random.default_rng(synth.config_seed(3) + 1)
    sizes = g.integers(40, 401, size=nslice)
    ks = np.concatenate([[200], 200 + np.cumsum(sizes)]).astype(np.int64)
    assert ks[-1] < n
    idx = np.unique(np.concatenate([ks, ks - 1]))
    lo, hi = pk.bisect(band, idx, rtol=1e-13, fanout=8)
    mid = dict(zip(idx.tolist(), (0.5 * (lo + hi)).tolist()))
    bounds = [0.5 * (mid[int(k) - 1] + mid[int(k)]) for k in ks]
    m0 = [oracle.m0_rule(int(c)) for c in sizes]
    lo2, hi2 = pk.bisect(band, [0, n - 1], rtol=1e-10, fanout=16)
    bnorm = max(abs(lo2[0]), abs(hi2[0]), abs(lo2[1]), abs(hi2[1]))
    X0 = synth.random_subspace(n, int(sum(m0)), synth.config_seed(3) + 2, False)
    r = pk.band_slice(band, bounds, m0, block_to_dev(X0, device), ne=ne, precision=pk.MIXED, bnorm=bnorm,
                      tol=1e-10, max_iter=40, hbm_cap_bytes=100 << 30, autotune=1, rr_arith=arith)
    assert r.status == 0
    assert r.stats["waves"] >= 2                      # the 1024 factorizations did not fit one group
    assert r.stats["factorizations"] == nslice * ne   # every system factored once (groups, not re-streaming)
    assert list(r.counts) == [int(c) for c in sizes]
    assert list(r.nfound) == list(r.counts)
    neg = [oracle.inertia(ab, s) for s in bounds]      # exact counts at all 65 boundaries
    assert list(np.diff(neg)) == [int(c) for c in sizes] == list(r.counts)
    ev = r.evals.cpu().numpy()
    off = np.concatenate([[0], np.cumsum(m0)])
    for i in (5, 40):                                 # residuals of two whole slices through the oracle
        k = int(r.nfound[i])
        Xi = r.evecs[off[i]: off[i] + k].cpu().numpy().T
        li = ev[off[i]: off[i] + k]
        assert np.max(oracle.residuals(ab, li, Xi, bnorm)) <= 1e-10
