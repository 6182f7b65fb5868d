"""GPU inertia (Sylvester counts by pivot-free LDL^T, Section 3.2) against the
oracle: counts and every pivot must be bit-identical."""
import numpy as np
import pytest

import oracle
import synth
from gpu_util import dev, to_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def device():
    return dev()


CASES = [(1, 0, False, 1), (2, 1, True, 2), (37, 3, True, 3), (200, 7, False, 4), (257, 32, False, 5),
         (300, 64, True, 6), (333, 128, True, 7), (150, 120, False, 8), (64, 63, True, 9), (500, 1, False, 10),
         # widest bands with the window in shared memory, and past it (window in the workspace)
         (420, 149, True, 11), (450, 194, False, 12), (400, 150, True, 13), (460, 195, False, 14),
         # n not above b: the window is the whole matrix
         (100, 149, True, 15)]


@pytest.mark.parametrize("n,b,cplx,seed", CASES)
def test_counts_and_pivots_bit_exact(device, n, b, cplx, seed):
    import paper_2012_00506_gb300 as pk
    ab = synth.random_band(n, b, 500 + seed, cplx)
    lo, hi = oracle.gershgorin(ab)
    rng = np.random.default_rng(seed)
    sig = np.concatenate([np.linspace(lo - 0.1, hi + 0.1, 7), rng.uniform(lo, hi, 5)])
    neg, piv = pk.inertia(to_dev(ab, device), sig, pivots=True)
    piv = piv.cpu().numpy()
    for s_i, s in enumerate(sig):
        c, d = oracle.inertia(ab, s, return_pivots=True)
        assert neg[s_i] == c
        assert np.array_equal(piv[s_i], d), (s_i, np.max(np.abs(piv[s_i] - d)))


def test_padded_leading_dimension(device):
    import paper_2012_00506_gb300 as pk
    ab = synth.random_band(120, 5, 77, True)
    abp = synth.pad_band(ab, 9)
    sig = [-0.3, 0.0, 0.41]
    assert list(pk.inertia(to_dev(abp, device), sig, b=5)) == [oracle.inertia(ab, s) for s in sig]


def test_laplacian_closed_form_full_size(device):
    import paper_2012_00506_gb300 as pk
    m, k = 63, 32
    ab = synth.laplacian_2d_band(m, k)
    i = np.arange(1, m + 1)[:, None]
    j = np.arange(1, k + 1)[None, :]
    ev = np.sort((4 - 2 * np.cos(i * np.pi / (m + 1)) - 2 * np.cos(j * np.pi / (k + 1))).ravel())
    u = np.unique(np.round(ev, 12))
    sig = 0.5 * (u[:-1] + u[1:])[::37]
    neg = pk.inertia(to_dev(ab, device), sig)
    assert all(neg[t] == np.sum(ev < s) for t, s in enumerate(sig))


def test_zero_pivot_rule(device):
    import paper_2012_00506_gb300 as pk
    d = np.array([0.5, -1.0, 2.0, -1.0, 0.0, 3.0])
    ab = synth.diagonal_band(d, 2)
    neg, piv = pk.inertia(to_dev(ab, device), [-1.0, 0.0], pivots=True)
    assert list(neg) == [oracle.inertia(ab, -1.0), oracle.inertia(ab, 0.0)] == [2, 3]
    assert np.sum(piv.cpu().numpy()[0] == -oracle.pivmin(ab)) == 2


def test_bisection_enclosures(device):
    import paper_2012_00506_gb300 as pk
    ab = synth.random_band(400, 9, 99, True)
    ev = np.linalg.eigvalsh(synth.band_to_dense(ab))
    idx = [0, 57, 200, 399]
    lo, hi = pk.bisect(to_dev(ab, device), idx, rtol=1e-13, fanout=8)
    for t, k in enumerate(idx):
        assert lo[t] <= ev[k] < hi[t] + 1e-15
        assert hi[t] - lo[t] <= 1e-13 * max(1.0, abs(lo[t]), abs(hi[t]))
        assert oracle.inertia(ab, lo[t]) <= k < oracle.inertia(ab, hi[t])
    # same FP64 operations in the same order on both sides: identical bits
    for ab2 in (ab, synth.random_band(301, 17, 98, False), synth.mixture_band(1000, 40, 97, is_complex=True)):
        glo, ghi = pk.gershgorin(to_dev(ab2, device))
        olo, ohi = oracle.gershgorin(ab2)
        assert (glo, ghi) == (olo, ohi), (glo - olo, ghi - ohi)
