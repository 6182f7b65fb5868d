"""GPU FEAST slicing (Algorithm 1 on every slice, behind pdeshep_band_slice)
against the oracle: exact counts, eigenvalues within 1e-10 ||B||_2, subspace
sines within 1e-8, residuals and orthogonality."""
import numpy as np
import pytest

import oracle
import synth
from gpu_util import block_from_dev, block_to_dev, dev, orth_tol, to_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def device():
    return dev()


def _bounds(ab, ks):
    return [oracle.boundary_between(ab, k) for k in ks]


def _run_compare(device, ab, ks, m0, precision, seed, ne=8, rho=0.3, tol=1e-10):
    import paper_2012_00506_gb300 as pk
    cplx = np.iscomplexobj(ab)
    n = ab.shape[0]
    bounds = _bounds(ab, ks)
    bnorm = oracle.spectral_norm(ab)
    X0 = synth.random_subspace(n, int(sum(m0)), seed, cplx)
    r = pk.band_slice(to_dev(ab, device), bounds, m0, block_to_dev(X0, device), ne=ne, precision=precision,
                      bnorm=bnorm, tol=tol, ellipse_ratio=rho, max_iter=40)
    assert r.status == 0, (r.status, r.stats)
    evals = r.evals.cpu().numpy()
    evecs = block_from_dev(r.evecs)
    off = 0
    for i in range(len(m0)):
        cnt = ks[i + 1] - ks[i]
        assert r.counts[i] == cnt == oracle.inertia(ab, bounds[i + 1]) - oracle.inertia(ab, bounds[i])
        assert r.nfound[i] == cnt
        o = oracle.feast_slice(ab, bounds[i], bounds[i + 1], X0[:, off:off + m0[i]], ne=ne, rho=rho, tol=tol,
                               bnorm=bnorm, max_iter=40, count=cnt)
        assert o["status"] == 0 and o["nfound"] == cnt
        lg = evals[off:off + cnt]
        Xg = evecs[:, off:off + cnt]
        assert np.max(np.abs(lg - o["evals"][:cnt])) <= 1e-10 * bnorm
        assert oracle.subspace_sin_angle(Xg, o["evecs"][:, :cnt]) <= 1e-8
        assert np.max(oracle.residuals(ab, lg, Xg, bnorm)) <= tol
        assert oracle.orth(Xg) < 1e-13
        # entrywise, without the 1/n: FP64 below 1e-13; mixed (tensor-core digit products by default)
        # within n u of its products' arithmetic
        assert oracle.orth_max(Xg) <= (1e-13 if precision == 0 else orth_tol(n, 2))
        off += m0[i]
    return r


@pytest.mark.parametrize("precision", [0, 1])
def test_real_one_slice(device, precision):
    ab = synth.random_band(300, 7, 21)
    _run_compare(device, ab, [120, 150], [oracle.m0_rule(30)], precision, 22)


@pytest.mark.parametrize("precision", [0, 1])
def test_complex_three_slices_uneven(device, precision):
    ab = synth.random_band(260, 6, 31, True)
    ks = [20, 30, 52, 90]
    m0 = [oracle.m0_rule(ks[i + 1] - ks[i]) for i in range(3)]
    _run_compare(device, ab, ks, m0, precision, 32)


def test_wide_band_ragged(device):
    ab = synth.random_band(333, 40, 41, True)
    _run_compare(device, ab, [100, 125], [35], 1, 42, ne=16, rho=1.0)


def test_laplacian_closed_form(device):
    import paper_2012_00506_gb300 as pk
    m, k = 26, 17
    ab = synth.laplacian_2d_band(m, k)
    i = np.arange(1, m + 1)[:, None]
    j = np.arange(1, k + 1)[None, :]
    ev = np.sort((4 - 2 * np.cos(i * np.pi / (m + 1)) - 2 * np.cos(j * np.pi / (k + 1))).ravel())
    lo, hi = 0.5 * (ev[99] + ev[100]), 0.5 * (ev[139] + ev[140])
    X0 = synth.random_subspace(m * k, 52, 5, False)
    r = pk.band_slice(to_dev(ab, device), [lo, hi], [52], block_to_dev(X0, device), ne=16, bnorm=float(ev[-1]),
                      tol=1e-11, ellipse_ratio=1.0)
    assert r.status == 0 and r.counts[0] == 40 and r.nfound[0] == 40
    assert np.max(np.abs(r.evals.cpu().numpy()[:40] - ev[100:140])) < 1e-11 * ev[-1]


def test_count_mismatch_and_nonfinite(device):
    import torch
    import paper_2012_00506_gb300 as pk
    ab = synth.random_band(200, 5, 51)
    b0, b1 = _bounds(ab, [10, 40])
    X0 = synth.random_subspace(200, 20, 52, False)
    r = pk.band_slice(to_dev(ab, device), [b0, b1], [20], block_to_dev(X0, device), raise_on_error=False)
    assert r.status == 2 and r.counts[0] == 30
    bad = ab.copy()
    bad[3, 1] = np.nan
    r = pk.band_slice(to_dev(bad, device), [b0, b1], [40], block_to_dev(synth.random_subspace(200, 40, 1, False),
                      device), raise_on_error=False)
    assert r.status == 4
    r = pk.band_slice(to_dev(ab, device), [b0, b1], [40], block_to_dev(synth.random_subspace(200, 40, 1, False),
                      device), max_iter=1, raise_on_error=False)
    assert r.status == 1


def test_streaming_waves_match_resident(device):
    import paper_2012_00506_gb300 as pk
    ab = synth.random_band(256, 8, 61, True)
    ks = [30, 45, 70]
    m0 = [25, 35]
    bounds = _bounds(ab, ks)
    bnorm = oracle.spectral_norm(ab)
    X0 = block_to_dev(synth.random_subspace(256, 60, 62, True), device)
    r1 = pk.band_slice(to_dev(ab, device), bounds, m0, X0, bnorm=bnorm)
    r2 = pk.band_slice(to_dev(ab, device), bounds, m0, X0, bnorm=bnorm, hbm_cap_bytes=3 << 20)
    assert r1.status == r2.status == 0
    assert r2.stats["waves"] > r1.stats["waves"]
    assert np.max(np.abs(r1.evals.cpu().numpy() - r2.evals.cpu().numpy())[:15]) < 1e-12


@pytest.mark.parametrize("cplx", [False, True])
def test_mixed_eigensolver_needs_no_fallback(device, cplx):
    """The FP32 Jacobi start plus FP64 refinement of the Rayleigh-Ritz eigenproblems
    converges on its own on a random band (every block refined, none sent to the FP64
    Jacobi path), and the slices still match the exact counts."""
    import paper_2012_00506_gb300 as pk
    n, b = 1500, 12
    ab = synth.random_band(n, b, 8080 + cplx, cplx)
    ks = [100, 260, 420]
    bounds = _bounds(ab, ks)
    m0 = [oracle.m0_rule(ks[i + 1] - ks[i]) for i in range(2)]
    X0 = synth.random_subspace(n, int(sum(m0)), 3, cplx)
    r = pk.band_slice(to_dev(ab, device), bounds, m0, block_to_dev(X0, device), precision=pk.MIXED,
                      bnorm=oracle.spectral_norm(ab), max_iter=30)
    assert r.status == 0
    assert list(r.nfound) == [ks[1] - ks[0], ks[2] - ks[1]]
    st = r.stats
    assert st["eig_refine_steps"] > 0
    assert st["eig_fallback_unconverged"] == 0 and st["eig_fallback_wide"] == 0, st
    assert st["jacobi_sweeps64"] == 0


def _small_problem(device, cplx, seed=77, n=1200, b=16, ks=(40, 160, 200, 460)):
    ab = synth.random_band(n, b, seed, cplx)
    bounds = _bounds(ab, list(ks))
    m0 = [oracle.m0_rule(ks[i + 1] - ks[i]) for i in range(len(ks) - 1)]   # uneven: 120+, 40+, 260+
    X0 = synth.random_subspace(n, int(sum(m0)), 4, cplx)
    return ab, bounds, m0, X0


@pytest.mark.parametrize("cplx", [False, True])
def test_rhs_block_width_does_not_change_results(device, cplx):
    """The persistent solves give the same bits for work items of 16, 32 or 64
    right-hand sides (each column's arithmetic is independent of the grouping), and the
    tensor-memory solve (128 columns, a thread per right-hand side) gives the same bits
    again: every entry is the same sequence of FP32 FMAs."""
    import paper_2012_00506_gb300 as pk
    ab, bounds, m0, X0 = _small_problem(device, cplx)
    band = to_dev(ab, device)
    outs = []
    for cw in (16, 32, 64, 128):
        r = pk.band_slice(band, bounds, m0, block_to_dev(X0, device), precision=pk.MIXED,
                          bnorm=oracle.spectral_norm(ab), rhs_chunk=cw, max_iter=30)
        assert r.status == 0 and r.stats["rhs_chunk_used"] == cw
        outs.append((r.evals.cpu().numpy(), r.evecs.cpu().numpy(), list(r.nfound)))
    for e, v, nf in outs[1:]:
        assert nf == outs[0][2]
        assert np.array_equal(e, outs[0][0]) and np.array_equal(v, outs[0][1])
    # the tensor-core solve (bf16x6 products: FP32-class, not the same FMA sequence) refines to the
    # same eigenpairs within the FEAST tolerances
    r = pk.band_slice(band, bounds, m0, block_to_dev(X0, device), precision=pk.MIXED,
                      bnorm=oracle.spectral_norm(ab), rhs_chunk=256, max_iter=30)
    assert r.status == 0 and r.stats["rhs_chunk_used"] == 256 and list(r.nfound) == outs[0][2]
    e = r.evals.cpu().numpy()
    bn = oracle.spectral_norm(ab)
    off = 0
    for i, m in enumerate(m0):
        k = int(r.nfound[i])
        assert np.max(np.abs(e[off:off + k] - outs[0][0][off:off + k])) <= 1e-11 * bn
        off += m


def test_uneven_slices_against_oracle(device):
    """Slices of 120, 40 and 260 eigenvalues in one batch (the uneven-m0 case the
    work queue balances) match the oracle slice by slice."""
    _run_compare(device, synth.random_band(1200, 16, 78, True), [40, 160, 200, 460],
                 [oracle.m0_rule(c) for c in (120, 40, 260)], 1, 21)


def test_autotuner_measures_then_reuses(device, tmp_path):
    """Float-float Rayleigh-Ritz products: the solve width and the Gram split are tuned once,
    stored, and reused from the file by a later process."""
    import paper_2012_00506_gb300 as pk
    ab, bounds, m0, X0 = _small_problem(device, True, seed=79)
    band = to_dev(ab, device)
    bn = oracle.spectral_norm(ab)
    cache = str(tmp_path / "tune.txt")
    pk.load().pdeshep_tune_reset()
    ff = dict(rr_arith=pk.RR_FLOATFLOAT)
    r1 = pk.band_slice(band, bounds, m0, block_to_dev(X0, device), bnorm=bn, autotune=2, tune_cache=cache, **ff)
    assert r1.status == 0 and r1.stats["tuned"] == 2
    cw, sp = r1.stats["rhs_chunk_used"], r1.stats["gram_splits_used"]
    assert cw in (16, 32, 64, 128) and sp in (2, 4, 8)
    # the tensor-core solve serves only the first passes, and only when it was measured faster
    early = r1.stats["rhs_chunk_early"]
    assert early in (0, 256)
    r2 = pk.band_slice(band, bounds, m0, block_to_dev(X0, device), bnorm=bn, autotune=1, tune_cache=cache, **ff)
    assert r2.stats["tuned"] == 0 and r2.stats["rhs_chunk_used"] == cw and r2.stats["gram_splits_used"] == sp
    assert r2.stats["rhs_chunk_early"] == early
    pk.load().pdeshep_tune_reset()          # in-process choices gone: the file still has them
    r3 = pk.band_slice(band, bounds, m0, block_to_dev(X0, device), bnorm=bn, autotune=1, tune_cache=cache, **ff)
    assert r3.stats["tuned"] == 0 and r3.stats["rhs_chunk_used"] == cw
    lines = open(cache).read().split("\n")
    assert any(l.startswith("solve/") for l in lines) and any(l.startswith("gram/") for l in lines)
    for r in (r1, r2, r3):
        assert list(r.nfound) == list(r.counts)
    assert np.allclose(r1.evals.cpu().numpy(), r3.evals.cpu().numpy(), rtol=0, atol=1e-11 * bn)


@pytest.mark.parametrize("cplx", [False, True])
def test_rr_arithmetics_agree(device, cplx):
    """Mixed precision with the Rayleigh-Ritz products in FP64, in float-float or as
    tensor-core digit products: each gives every in-slice eigenvalue within 1e-10 ||B||
    of the dense spectrum, residuals <= 1e-10 and orthonormal vectors, and they agree
    with each other to 1e-11 ||B|| (each run stops at its own iterate once the
    residuals pass 1e-10, so they are not expected to agree further)."""
    import paper_2012_00506_gb300 as pk
    ab, bounds, m0, X0 = _small_problem(device, cplx, seed=80)
    band = to_dev(ab, device)
    bn = oracle.spectral_norm(ab)
    res = {}
    ariths = (pk.RR_FLOATFLOAT, pk.RR_FP64, pk.RR_TENSOR)
    for arith in ariths:
        r = pk.band_slice(band, bounds, m0, block_to_dev(X0, device), bnorm=bn, rr_arith=arith, max_iter=30)
        assert r.status == 0 and list(r.nfound) == list(r.counts)
        res[arith] = r
    ev = np.linalg.eigvalsh(synth.band_to_dense(ab))
    off = 0
    for i, m in enumerate(m0):
        k = int(res[pk.RR_FP64].nfound[i])
        truth = ev[(ev >= bounds[i]) & (ev < bounds[i + 1])]
        vals = {a: res[a].evals.cpu().numpy()[off:off + k] for a in ariths}
        for a in ariths:
            assert np.max(np.abs(np.sort(vals[a]) - truth)) <= 1e-10 * bn
            assert np.max(np.abs(vals[a] - vals[pk.RR_FP64])) <= 1e-11 * bn
        X = block_from_dev(res[pk.RR_TENSOR].evecs)[:, off:off + k]
        assert np.max(oracle.residuals(ab, vals[pk.RR_TENSOR], X, bn)) <= 1e-10
        assert oracle.orth(X) < 1e-13
        off += m


@pytest.mark.parametrize("cplx", [False, True])
def test_graph_replay_matches_direct_launches(device, cplx):
    """Filter passes replayed from CUDA graphs give the same bits as direct launches."""
    import torch
    import paper_2012_00506_gb300 as pk
    ab, bounds, m0, X0 = _small_problem(device, cplx, seed=81)
    band = to_dev(ab, device)
    bn = oracle.spectral_norm(ab)
    s = torch.cuda.Stream()
    outs = []
    with torch.cuda.stream(s):
        for graphs in (0, 1):
            r = pk.band_slice(band, bounds, m0, block_to_dev(X0, device), bnorm=bn, graphs=graphs, stream=s,
                              rhs_chunk=32, max_iter=30)
            s.synchronize()
            assert r.status == 0 and list(r.nfound) == list(r.counts)
            outs.append(r)
    assert outs[0].stats["graph_launches"] == 0 and outs[1].stats["graph_launches"] >= 1
    assert outs[0].stats["iterations"] == outs[1].stats["iterations"]
    assert np.array_equal(outs[0].evals.cpu().numpy(), outs[1].evals.cpu().numpy())
    assert np.array_equal(outs[0].evecs.cpu().numpy(), outs[1].evecs.cpu().numpy())


def test_random_start_matches_oracle_stream(device):
    """pdeshep_random_start writes exactly the oracle's counter-based start vectors."""
    import paper_2012_00506_gb300 as pk
    for cplx in (False, True):
        X = pk.random_start(300, 17, cplx, seed=99, col0=5, device=device)
        ref = oracle.random_start(300, 17, cplx, seed=99, col0=5)
        assert np.array_equal(block_from_dev(X), ref)


@pytest.mark.parametrize("cplx", [False, True])
def test_library_drawn_start_vectors(device, cplx):
    """d_x0 = NULL: the library draws the start vectors of Algorithm 1 itself.  The run gives the
    same bits as one handed the oracle's copy of that stream, and matches the oracle's FEAST
    started from those vectors."""
    import paper_2012_00506_gb300 as pk
    n, b = 500, 9
    ab = synth.random_band(n, b, 301 + cplx, cplx)
    ks = [60, 100, 130]
    bounds = _bounds(ab, ks)
    m0 = [oracle.m0_rule(40), oracle.m0_rule(30)]
    bn = oracle.spectral_norm(ab)
    band = to_dev(ab, device)
    r0 = pk.band_slice(band, bounds, m0, None, seed=1234, bnorm=bn, max_iter=40)
    X0 = oracle.random_start(n, sum(m0), cplx, seed=1234)
    r1 = pk.band_slice(band, bounds, m0, block_to_dev(X0, device), bnorm=bn, max_iter=40)
    assert r0.status == r1.status == 0
    assert np.array_equal(r0.evals.cpu().numpy(), r1.evals.cpu().numpy())
    assert np.array_equal(r0.evecs.cpu().numpy(), r1.evecs.cpu().numpy())
    ev, V = r0.evals.cpu().numpy(), block_from_dev(r0.evecs)
    off = 0
    for i in range(2):
        cnt = ks[i + 1] - ks[i]
        assert r0.counts[i] == r0.nfound[i] == cnt
        o = oracle.feast_slice(ab, bounds[i], bounds[i + 1], X0[:, off:off + m0[i]], ne=8, tol=1e-10, bnorm=bn,
                               max_iter=40, count=cnt)
        assert o["status"] == 0 and o["nfound"] == cnt
        assert np.max(np.abs(ev[off:off + cnt] - o["evals"][:cnt])) <= 1e-10 * bn
        assert oracle.subspace_sin_angle(V[:, off:off + cnt], o["evecs"][:, :cnt]) <= 1e-8
        off += m0[i]


@pytest.mark.parametrize("cplx", [False, True])
def test_m0_resize_enlarges_small_subspaces(device, cplx):
    """m0_resize (Section 3.2's subspace rule in the library): slice 0 is given 12 columns for
    40 eigenvalues and runs with max(ceil(1.3 * 40), 40 + 10) = 52; slices whose m0 already
    covers m_i + 10 keep theirs.  Every slice ends with its exact count and matches the oracle
    started from the same columns.  Without the option the same call reports the mismatch, and
    a capacity below a count is a mismatch too."""
    import paper_2012_00506_gb300 as pk
    n, b = 600, 10
    ab = synth.random_band(n, b, 401 + cplx, cplx)
    ks = [50, 90, 100, 160]
    counts = [40, 10, 60]
    bounds = _bounds(ab, ks)
    bn = oracle.spectral_norm(ab)
    band = to_dev(ab, device)
    m0, cap = [12, 30, 70], 80
    X0 = oracle.random_start(n, 3 * cap, cplx, seed=5)
    r = pk.band_slice(band, bounds, m0, block_to_dev(X0, device), bnorm=bn, m0_resize=1, m0_cap=cap, max_iter=40)
    assert r.status == 0
    assert list(r.m0) == [52, 30, 70]
    assert list(r.counts) == counts and list(r.nfound) == counts
    ev, V = r.evals.cpu().numpy(), block_from_dev(r.evecs)
    for i in range(3):
        off, cnt = i * cap, counts[i]
        o = oracle.feast_slice(ab, bounds[i], bounds[i + 1], X0[:, off:off + int(r.m0[i])], ne=8, tol=1e-10,
                               bnorm=bn, max_iter=40, count=cnt)
        assert o["status"] == 0 and o["nfound"] == cnt
        assert np.max(np.abs(ev[off:off + cnt] - o["evals"][:cnt])) <= 1e-10 * bn
        assert oracle.subspace_sin_angle(V[:, off:off + cnt], o["evecs"][:, :cnt]) <= 1e-8
    r2 = pk.band_slice(band, bounds, m0, None, bnorm=bn, raise_on_error=False)
    assert r2.status == 2 and list(r2.counts) == counts
    r3 = pk.band_slice(band, bounds, [12, 30, 30], None, bnorm=bn, m0_resize=1, m0_cap=35, raise_on_error=False)
    assert r3.status == 2 and list(r3.counts) == counts and list(r3.m0) == [35, 30, 35]
    r4 = pk.band_slice(band, bounds, m0, None, bnorm=bn, m0_resize=1, m0_cap=35, raise_on_error=False)
    assert r4.status == -11                              # a given m0 above the capacity is an argument error


def test_slice_groups_match_one_batch(device):
    """A factor cap that holds slices 0-1 but not slice 2 as well: the call runs as two groups,
    each factoring its systems once and iterating on resident factors, with the results of the
    single batch (and exact counts)."""
    import paper_2012_00506_gb300 as pk
    ab, bounds, m0, X0 = _small_problem(device, True, seed=82)
    band = to_dev(ab, device)
    bn = oracle.spectral_norm(ab)
    r1 = pk.band_slice(band, bounds, m0, block_to_dev(X0, device), bnorm=bn, max_iter=30)
    # per system (n = 1200, b = 16, complex64): 1.87 MB of factors + n m0 x 2 solve outputs;
    # slices 0 + 1 need 61.9 MB for their 16 systems, slice 2 alone 66.9 MB
    r2 = pk.band_slice(band, bounds, m0, block_to_dev(X0, device), bnorm=bn, max_iter=30, hbm_cap_bytes=70_000_000)
    assert r1.status == r2.status == 0
    assert r1.stats["waves"] == 1 and r2.stats["waves"] == 2
    assert r2.stats["factorizations"] == r1.stats["factorizations"] == 8 * 3
    assert list(r2.counts) == list(r1.counts) and list(r2.nfound) == list(r1.nfound) == list(r1.counts)
    e1, e2 = r1.evals.cpu().numpy(), r2.evals.cpu().numpy()
    off = 0
    for i, m in enumerate(m0):
        k = int(r1.nfound[i])
        assert np.max(np.abs(e1[off:off + k] - e2[off:off + k])) <= 1e-12 * bn
        off += m


def test_zolotarev_rule_through_gpu_feast(device):
    """The Zolotarev rule (the rational filter Section 2.2 cites after eq. (10)) from the library's
    host code, passed as the call's nodes and weights: the GPU FEAST matches the oracle's FEAST run
    with the oracle's own Zolotarev rule."""
    import paper_2012_00506_gb300 as pk
    from oracle import rules_oracle
    n, b = 400, 8
    ab = synth.random_band(n, b, 503, True)
    ks = [90, 130, 170]
    bounds = _bounds(ab, ks)
    bn = oracle.spectral_norm(ab)
    m0 = [oracle.m0_rule(40), oracle.m0_rule(40)]
    rules = [rules_oracle.zolotarev_rule(8, bounds[i], bounds[i + 1], 0.1)[:2] for i in range(2)]
    lib_rules = [pk.zolotarev_rule(8, bounds[i], bounds[i + 1], 0.1)[:2] for i in range(2)]
    for (z, w), (zl, wl) in zip(rules, lib_rules):
        assert np.max(np.abs(z - zl)) <= 1e-12 * bn and np.max(np.abs(w - wl)) <= 1e-12 * np.max(np.abs(w))
    X0 = synth.random_subspace(n, sum(m0), 504, True)
    r = pk.band_slice(to_dev(ab, device), bounds, m0, block_to_dev(X0, device), bnorm=bn, max_iter=40,
                      nodes=np.concatenate([z for z, _ in lib_rules]), weights=np.concatenate([w for _, w in lib_rules]))
    assert r.status == 0
    ev, V = r.evals.cpu().numpy(), block_from_dev(r.evecs)
    off = 0
    for i in range(2):
        cnt = ks[i + 1] - ks[i]
        assert r.counts[i] == r.nfound[i] == cnt
        o = oracle.feast_slice(ab, bounds[i], bounds[i + 1], X0[:, off:off + m0[i]], tol=1e-10, bnorm=bn,
                               max_iter=40, count=cnt, rule=rules[i])
        assert o["status"] == 0 and o["nfound"] == cnt
        assert np.max(np.abs(ev[off:off + cnt] - o["evals"][:cnt])) <= 1e-10 * bn
        assert oracle.subspace_sin_angle(V[:, off:off + cnt], o["evecs"][:, :cnt]) <= 1e-8
        assert oracle.orth_max(V[:, off:off + cnt]) <= orth_tol(n, 2)
        off += m0[i]


def test_trapezoid_rule_through_gpu_feast(device):
    """The midpoint trapezoid rule (Section 2.2 names it beside Gauss quadrature) passed as the
    call's nodes and weights: the GPU FEAST matches the oracle's FEAST run with the same rule."""
    import paper_2012_00506_gb300 as pk
    from oracle import rules_oracle
    n, b = 400, 8
    ab = synth.random_band(n, b, 501, True)
    ks = [100, 140, 175]
    bounds = _bounds(ab, ks)
    bn = oracle.spectral_norm(ab)
    m0 = [oracle.m0_rule(40), oracle.m0_rule(35)]
    rules = [rules_oracle.trapezoid_rule(8, bounds[i], bounds[i + 1], 0.3) for i in range(2)]
    lib_rules = [pk.contour_rule(8, bounds[i], bounds[i + 1], 0.3, kind="trapezoid") for i in range(2)]
    for (z, w), (zl, wl) in zip(rules, lib_rules):
        assert np.allclose(z, zl, rtol=0, atol=1e-15) and np.allclose(w, wl, rtol=0, atol=1e-15)
    X0 = synth.random_subspace(n, sum(m0), 502, True)
    r = pk.band_slice(to_dev(ab, device), bounds, m0, block_to_dev(X0, device), bnorm=bn, max_iter=40,
                      nodes=np.concatenate([z for z, _ in lib_rules]), weights=np.concatenate([w for _, w in lib_rules]))
    assert r.status == 0
    ev, V = r.evals.cpu().numpy(), block_from_dev(r.evecs)
    off = 0
    for i in range(2):
        cnt = ks[i + 1] - ks[i]
        assert r.counts[i] == r.nfound[i] == cnt
        o = oracle.feast_slice(ab, bounds[i], bounds[i + 1], X0[:, off:off + m0[i]], tol=1e-10, bnorm=bn,
                               max_iter=40, count=cnt, rule=rules[i])
        assert o["status"] == 0 and o["nfound"] == cnt
        assert np.max(np.abs(ev[off:off + cnt] - o["evals"][:cnt])) <= 1e-10 * bn
        assert oracle.subspace_sin_angle(V[:, off:off + cnt], o["evecs"][:, :cnt]) <= 1e-8
        assert oracle.orth_max(V[:, off:off + cnt]) <= orth_tol(n, 2)
        off += m0[i]
