"""GPU slice proposer against the oracle: features, network forward/gradient,
Adam step, and the proposal's exact counts (inertia, Section 3.2) with its
multisection fall-back; plus the gain of a trained network over equal-width
slicing (the equal-width partition the paper compares its balanced slicing
with, Section 3.1)."""
import numpy as np
import pytest

import oracle
import synth
from gpu_util import dev, to_dev
from oracle import slicer_oracle as so

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def device():
    return dev()


@pytest.mark.parametrize("n,b,cplx,seed", [(1000, 8, False, 1), (3001, 20, True, 2), (64, 0, False, 3),
                                           (513, 63, True, 4)])
def test_features_vs_oracle(device, n, b, cplx, seed):
    from paper_2012_00506_gb300 import slicer
    ab = synth.mixture_band(n, b, 40 + seed, is_complex=cplx, off_sigma=0.05)
    f = slicer.features(to_dev(ab, device), seed=1234 + seed).cpu().numpy().astype(np.float64)
    g = so.features(ab, 1234 + seed)
    # histogram: the Gershgorin interval and every bin decision are the same FP64 operations
    # in the same order on both sides, so the bin counts are identical
    assert np.array_equal(f[:64].astype(np.float32), g[:64].astype(np.float32)), (f[:64] * n, g[:64] * n)
    assert np.array_equal(np.rint(f[:64].astype(np.float64) * n), np.rint(g[:64] * n))
    assert np.allclose(f[64:66], g[64:66], rtol=1e-6, atol=1e-7)
    assert np.allclose(f[66:], g[66:], rtol=0, atol=2e-7), np.abs(f[66:] - g[66:]).max()


def _params(seed, device):
    from paper_2012_00506_gb300 import slicer
    return slicer.init_params(seed, device, last_scale=1.0)


def test_forward_vs_oracle(device):
    import torch
    from paper_2012_00506_gb300 import slicer
    p = _params(3, device)
    X = torch.from_numpy(np.random.default_rng(0).normal(size=(45, 98)).astype(np.float32)).to(device)
    c = slicer.mlp_forward(p, X).cpu().numpy()
    co = so.forward(p.cpu().numpy().astype(np.float64), X.cpu().numpy().astype(np.float64))
    assert np.abs(c - co).max() < 2e-5
    assert np.all(np.diff(c, axis=1) >= 0)


@pytest.mark.parametrize("batch", [1, 37, 64])
def test_gradient_vs_oracle(device, batch):
    import torch
    from paper_2012_00506_gb300 import slicer
    p = _params(5 + batch, device)
    g_ = np.random.default_rng(batch)
    X = torch.from_numpy(g_.normal(size=(batch, 98)).astype(np.float32)).to(device)
    T = torch.from_numpy(np.sort(g_.uniform(size=(batch, 63)), axis=1).astype(np.float32)).to(device)
    grad, loss = slicer.mlp_grad(p, X, T)
    lo, go = so.loss_and_grad(p.cpu().numpy().astype(np.float64), X.cpu().numpy().astype(np.float64),
                              T.cpu().numpy().astype(np.float64))
    gg = grad.cpu().numpy().astype(np.float64)
    assert abs(float(loss.item()) - lo) <= 1e-5 * lo
    assert np.linalg.norm(gg - go) <= 1e-4 * np.linalg.norm(go)
    # per layer too, so that a small layer's error is not hidden by the others
    for wo, bo, fo, fi in slicer.layer_offsets():
        for a, z in ((wo, wo + fo * fi), (bo, bo + fo)):
            assert np.linalg.norm(gg[a:z] - go[a:z]) <= 1e-4 * np.linalg.norm(go[a:z]) + 1e-9


def test_adam_step_vs_oracle(device):
    import torch
    from paper_2012_00506_gb300 import slicer
    p = _params(9, device)
    p0 = p.cpu().numpy().astype(np.float64)
    g_ = np.random.default_rng(9)
    X = torch.from_numpy(g_.normal(size=(16, 98)).astype(np.float32)).to(device)
    T = torch.from_numpy(np.sort(g_.uniform(size=(16, 63)), axis=1).astype(np.float32)).to(device)
    tr = slicer.Trainer(p, lr=1e-3, max_batch=16)
    _, go = so.loss_and_grad(p0, X.cpu().numpy().astype(np.float64), T.cpu().numpy().astype(np.float64))
    tr.step(X, T)
    p1 = tr.params.cpu().numpy().astype(np.float64)
    po, _, _ = so.adam_step(p0, go, np.zeros_like(p0), np.zeros_like(p0), 1, 1e-3)
    # step 1 moves every parameter by about lr * sign(g); compare where the sign is well determined
    sure = np.abs(go) > 1e-2 * np.sqrt(np.mean(go ** 2))
    assert sure.mean() > 0.5
    assert np.abs((p1 - p0)[sure] - (po - p0)[sure]).max() < 2e-5


def _check_counts(ab, pr, frac, nslices, tol, exact_targets=True):
    n = ab.shape[0]
    bd = pr.bounds
    assert np.all(np.diff(bd) >= 0)
    neg = [oracle.inertia(ab, s) for s in bd]
    assert np.array_equal(np.diff(neg), pr.counts), (np.diff(neg), pr.counts)
    tgt = np.floor(n * (frac[0] + (frac[1] - frac[0]) * np.arange(nslices + 1) / nslices) + 0.5).astype(int)
    if exact_targets:
        assert np.all(np.abs(np.array(neg) - tgt) <= tol), (neg, tgt)
    return np.array(neg), tgt


@pytest.mark.parametrize("cplx,frac,nslices,tol", [(False, (0.0, 1.0), 16, 0), (True, (0.1, 0.4), 12, 3),
                                                  (False, (0.0, 0.3), 7, 1), (True, (0.5, 1.0), 1, 0)])
def test_proposal_counts_exact_without_network(device, cplx, frac, nslices, tol):
    from paper_2012_00506_gb300 import slicer
    ab = synth.mixture_band(700, 9, 71, is_complex=cplx, off_sigma=0.03)
    pr = slicer.propose_slices(to_dev(ab, device), None, nslices=nslices, frac=frac, count_tol=tol)
    _check_counts(ab, pr, frac, nslices, tol)
    assert pr.inertia_evals >= nslices - 1


def test_proposal_cluster_wider_than_tolerance(device):
    """Eigenvalue 1.0 with multiplicity 40: a boundary inside it cannot reach its target;
    the closest exact count is kept and all counts stay exact."""
    from paper_2012_00506_gb300 import slicer
    d = np.concatenate([np.linspace(-2, 0, 60), np.full(40, 1.0), np.linspace(2, 3, 28)])
    ab = synth.diagonal_band(d, 2)
    pr = slicer.propose_slices(to_dev(ab, device), None, nslices=8, count_tol=0)
    neg, tgt = _check_counts(ab, pr, (0.0, 1.0), 8, 0, exact_targets=False)
    assert neg[0] == 0 and neg[-1] == 128 and pr.counts.sum() == 128
    for k in range(9):
        if not (60 < tgt[k] < 100):                  # targets outside the cluster are met exactly
            assert neg[k] == tgt[k]
        else:
            assert neg[k] in (60, 100)


def _family(seed, n, b):
    """Clustered spectra: Gaussian mixtures with random centres, widths and weights."""
    g = np.random.default_rng(seed)
    k = int(g.integers(1, 7))
    means = g.uniform(-1.0, 1.0, size=k)
    w = g.dirichlet(np.ones(k))
    return synth.mixture_band(n, b, seed, ncomp=k, comp_sigma=float(g.uniform(0.01, 0.2)),
                              off_sigma=float(g.uniform(0.005, 0.03)), means=means, weights=w)


@pytest.fixture(scope="module")
def trained(device):
    from paper_2012_00506_gb300 import slicer
    bands = [to_dev(_family(1000 + s, 1024, 8), device) for s in range(1024)]
    params, losses, _ = slicer.train(bands, steps=3000, batch=64, lr=1e-3, seed=0, log_every=250)
    return params, losses


def test_training_reduces_loss(trained):
    _, losses = trained
    assert losses[-1][1] < 0.1 * losses[0][1], losses


@pytest.mark.parametrize("tol", [4, 16])
def test_network_gain_over_equal_widths(device, trained, tol):
    """Held-out spectra of the same family: the trained network's boundaries are much
    closer in count to the equal-count targets than equal widths, and the proposal
    needs fewer inertia evaluations in all; counts are exact either way."""
    from paper_2012_00506_gb300 import slicer
    params, _ = trained
    err = {"mlp": [], "none": []}
    evals = {"mlp": 0, "none": 0}
    for s in range(16):
        ab = _family(50000 + s, 1024, 8)
        band = to_dev(ab, device)
        tgt = np.floor(1024 * np.arange(17) / 16 + 0.5).astype(int)
        for name, p in (("mlp", params), ("none", None)):
            pr = slicer.propose_slices(band, p, nslices=16, count_tol=tol)
            if s < 4:
                _check_counts(ab, pr, (0.0, 1.0), 16, tol)
            err[name] += list(np.abs(pr.proposed_counts - tgt)[1:-1])
            evals[name] += pr.inertia_evals
    e_m, e_u = np.mean(err["mlp"]), np.mean(err["none"])
    print(f"\nproposal count error (tol {tol}): network {e_m:.1f}, equal widths {e_u:.1f}; "
          f"inertia evaluations: network {evals['mlp']}, equal widths {evals['none']}")
    assert e_m < 0.33 * e_u, (e_m, e_u, evals)
    assert evals["mlp"] < evals["none"], (e_m, e_u, evals)


def test_weights_roundtrip(device, trained, tmp_path):
    from paper_2012_00506_gb300 import slicer
    params, _ = trained
    path = str(tmp_path / "slicer")
    slicer.save_params(path, params, {"family": "gaussian mixtures n=1024 b=8"})
    q, head = slicer.load_params(path, device)
    assert head["param_count"] == slicer.param_count()
    assert np.array_equal(q.cpu().numpy(), params.cpu().numpy())


def test_proposal_full_size_complex(device, trained):
    """n = 16384, b = 64 complex, 63 boundaries: counts at sampled boundaries equal the oracle's."""
    from paper_2012_00506_gb300 import slicer
    params, _ = trained
    ab = synth.mixture_band(16384, 64, 4242, is_complex=True, off_sigma=0.01)
    pr = slicer.propose_slices(to_dev(ab, device), params, nslices=64, count_tol=16)
    assert pr.counts.sum() == 16384 and np.all(np.diff(pr.bounds) >= 0)
    cum = np.concatenate([[0], np.cumsum(pr.counts)])
    for k in (1, 20, 47, 63):
        assert oracle.inertia(ab, pr.bounds[k]) == cum[k]
        assert abs(cum[k] - 16384 * k // 64) <= 16


@pytest.mark.parametrize("n,b,cplx,nsl", [(400, 12, True, 64), (257, 5, False, 16)])
def test_equal_count_targets_vs_oracle(device, n, b, cplx, nsl):
    """The training labels come from the library (bisection on inertia, Gershgorin
    normalisation): within rounding of the oracle's labels from the exact spectrum."""
    from paper_2012_00506_gb300 import slicer
    ab = synth.mixture_band(n, b, 70 + n, is_complex=cplx, off_sigma=0.03)
    t = slicer.equal_count_targets(to_dev(ab, device), nslices=nsl, rtol=1e-12)
    ref = so.equal_count_targets(ab, nsl)
    assert t.dtype == np.float32 and t.shape == (nsl - 1,)
    assert np.max(np.abs(t.astype(np.float64) - ref)) <= 2e-7
    assert np.all(np.diff(t) >= 0)
