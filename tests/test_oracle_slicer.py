"""Pins for the oracle of the learned slice proposer.

The proposer is not in the paper (it follows the density-of-states remark of
Section 3.1 and the equal-count objective of Section 3.1); what is pinned here
is the arithmetic it is built from: the SplitMix64 probe generator (published
outputs), the histogram and Chebyshev moments (closed forms on diagonal bands,
an eigendecomposition route on general bands, scale/shift invariances), the
network's gradient (central finite differences) and Adam's first step (closed
form).
"""
import os

import numpy as np
import pytest

import oracle
import synth
from oracle import slicer_oracle as so

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_splitmix64_published_outputs():
    rows = [ln.split() for ln in open(os.path.join(GOLDEN, "splitmix64.txt")) if not ln.startswith("#")]
    assert len(rows) == 3
    for _, state, out in rows:
        assert so.splitmix64(int(state, 16)) == int(out, 16)


def test_probes_are_rademacher_and_seeded():
    Z = so.probes(500, 7)
    assert Z.shape == (500, 8)
    assert set(np.unique(Z)) == {-1.0, 1.0}
    assert abs(Z.mean()) < 0.1                      # 4000 fair signs: std 0.016
    assert np.array_equal(Z, so.probes(500, 7))
    assert not np.array_equal(Z, so.probes(500, 8))
    # entry (i, p) depends on seed + p n + i only: shifting the seed by n shifts the probes by one column
    Z2 = so.probes(500, 7 + 500)
    assert np.array_equal(Z2[:, :7], Z[:, 1:])


def test_histogram_bin_centres():
    lo, hi = -2.0, 6.0
    w = (hi - lo) / 64
    ks = np.array([0, 0, 5, 63, 63, 63, 31, 32])
    d = lo + (ks + 0.5) * w
    d = np.concatenate([d, [lo - 1.0, hi + 5.0]])   # out of range: clamp to the end bins
    h = so.histogram(d, lo, hi)
    expect = np.zeros(64)
    for k in list(ks) + [0, 63]:
        expect[k] += 1
    assert np.array_equal(h, expect / d.size)


def _cheb(k, x):
    return np.cos(k * np.arccos(np.clip(x, -1.0, 1.0)))


@pytest.mark.parametrize("cplx", [False, True])
def test_moments_diagonal_closed_form(cplx):
    rng = np.random.default_rng(3)
    d = rng.uniform(-3.0, 5.0, size=300)
    ab = synth.diagonal_band(d, 4, is_complex=cplx)
    lo, hi = oracle.gershgorin(ab)
    assert (lo, hi) == (d.min(), d.max())
    f = so.features(ab, seed=11)
    x = (d - 0.5 * (lo + hi)) / (0.5 * (hi - lo))
    # z_i^2 = 1, so z^T T_k(D) z = sum_i T_k(x_i) for every probe
    mu = np.array([np.mean(_cheb(k, x)) for k in range(32)])
    assert np.allclose(f[66:], mu, atol=1e-12, rtol=0)
    s = max(abs(lo), abs(hi))
    assert f[64] == pytest.approx(0.5 * (lo + hi) / s) and f[65] == pytest.approx(0.5 * (hi - lo) / s)
    assert f[:64].sum() == pytest.approx(1.0)


@pytest.mark.parametrize("cplx", [False, True])
def test_moments_by_eigendecomposition(cplx):
    n, b = 120, 5
    ab = synth.random_band(n, b, seed=21, is_complex=cplx, off_sigma=0.3)
    lo, hi = oracle.gershgorin(ab)
    c, r = 0.5 * (lo + hi), 0.5 * (hi - lo)
    lam, V = np.linalg.eigh(synth.band_to_dense(ab))
    x = (lam - c) / r
    assert np.all(np.abs(x) <= 1.0)                  # Gershgorin encloses the spectrum
    Z = so.probes(n, 99)
    W = V.conj().T @ Z                                # probe coordinates in the eigenbasis
    mu = np.array([np.sum(_cheb(k, x)[:, None] * np.abs(W) ** 2) / (n * 8) for k in range(32)])
    f = so.features(ab, seed=99)
    assert np.allclose(f[66:], mu, atol=1e-11, rtol=0)


def test_features_scale_and_shift_invariance():
    ab = synth.mixture_band(200, 6, seed=5, off_sigma=0.05)
    f = so.features(ab, seed=1)
    g = so.features(3.5 * ab, seed=1)
    assert np.allclose(f, g, atol=1e-12, rtol=0)      # all 98 features are scale-free
    sh = ab.copy()
    sh[:, 0] += 10.0
    h = so.features(sh, seed=1)
    assert np.allclose(h[:64], f[:64], atol=0) or np.abs(h[:64] - f[:64]).sum() <= 2.0 / 200
    assert np.allclose(h[66:], f[66:], atol=1e-10)   # moments see only the scaled band
    assert h[64] != pytest.approx(f[64])             # the centre moves with the shift
    assert np.allclose(f[:64].sum(), 1.0)


def _rand_params(seed, scale=1.0):
    g = np.random.default_rng(seed)
    parts = []
    for l in range(4):
        fi, fo = so.DIMS[l], so.DIMS[l + 1]
        parts.append(g.normal(0, scale * np.sqrt(2.0 / fi), size=fo * fi))
        parts.append(g.normal(0, 0.1, size=fo))
    return np.concatenate(parts)


def test_zero_network_proposes_equal_widths():
    p = np.zeros(sum(so.DIMS[l] * so.DIMS[l + 1] + so.DIMS[l + 1] for l in range(4)))
    X = np.random.default_rng(0).normal(size=(3, 98))
    c = so.forward(p, X)
    assert c.shape == (3, 63)
    assert np.allclose(c, np.arange(1, 64)[None, :] / 64.0, atol=1e-15)


def test_forward_monotone_and_loss_zero_at_own_output():
    p = _rand_params(1)
    X = np.random.default_rng(2).normal(size=(5, 98))
    c = so.forward(p, X)
    assert np.all(np.diff(c, axis=1) > 0) and np.all(c > 0) and np.all(c < 1)
    loss, g = so.loss_and_grad(p, X, c)
    assert loss == 0.0 and np.all(g == 0.0)


def test_gradient_central_differences():
    p = _rand_params(4)
    g_ = np.random.default_rng(5)
    X = g_.normal(size=(6, 98))
    T = np.sort(g_.uniform(size=(6, 63)), axis=1)
    loss, grad = so.loss_and_grad(p, X, T)
    assert grad.shape == p.shape
    # a sample of parameters in every layer, weights and biases
    offs, idx = 0, []
    for l in range(4):
        fi, fo = so.DIMS[l], so.DIMS[l + 1]
        idx += list(offs + g_.choice(fo * fi, 12, replace=False))
        idx += list(offs + fo * fi + g_.choice(fo, 4, replace=False))
        offs += fo * fi + fo
    h = 1e-5
    for i in idx:
        pp, pm = p.copy(), p.copy()
        pp[i] += h
        pm[i] -= h
        fd = (so.loss_and_grad(pp, X, T)[0] - so.loss_and_grad(pm, X, T)[0]) / (2 * h)
        assert abs(fd - grad[i]) <= 1e-6 * max(abs(grad[i]), 1e-4 * np.abs(grad).max()), (i, fd, grad[i])


def test_adam_first_step_closed_form():
    g_ = np.random.default_rng(6)
    p = g_.normal(size=50)
    g = g_.normal(size=50)
    lr = 1e-3
    p1, m, v = so.adam_step(p, g, np.zeros(50), np.zeros(50), 1, lr)
    # bias-corrected moments of step 1 are g and g^2
    assert np.allclose(p1, p - lr * g / (np.abs(g) + 1e-8), rtol=0, atol=1e-15)
    assert np.allclose(m, 0.1 * g) and np.allclose(v, 0.001 * g * g)
