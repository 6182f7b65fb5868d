"""Pins of the partitioning oracle (Algorithm 3, Approach-1/-2 and Algorithm 4 of the paper,
Sections 3.1-3.2) against facts that do not come from the oracle itself: cluster structure
built into the data, exact invariances, counting identities, and closed-form spectra."""
import numpy as np
import pytest

import oracle
import synth
from oracle import partition_oracle as po


def _clusters(sizes, centers, width, seed):
    g = np.random.default_rng(seed)
    return np.sort(np.concatenate([c + width * g.standard_normal(s) for c, s in zip(centers, sizes)]))


@pytest.mark.parametrize("sizes,centers", [([30, 50, 20, 40], [0.0, 1.0, 2.5, 3.0]),
                                           ([10, 40, 25, 60, 15], [0.0, 2.0, 4.0, 6.0, 8.0]),
                                           ([12, 90, 8, 45, 30], [-3.0, -1.0, 1.5, 2.5, 6.0])])
def test_kmeans_recovers_separated_clusters(sizes, centers):
    """Well-separated clusters of unequal size: the equal-count start cuts through them, the
    k-means sweeps move every boundary into a gap between clusters."""
    d = _clusters(sizes, centers, 0.01, 11)
    b, c, sweeps = po.kmeans_slices(d, len(sizes), d[0] - 1, d[-1] + 1)
    assert c == sizes
    assert sweeps < 50
    ends = np.cumsum(sizes)
    for i, e in enumerate(ends[:-1]):
        assert d[e - 1] < b[i + 1] < d[e]            # the boundary sits in the gap
    _, c1 = po.equal_count_slices(d, len(sizes), d[0] - 1, d[-1] + 1)
    assert c1 != sizes


def test_equal_counts_and_widths():
    d = np.sort(np.random.default_rng(2).uniform(-1, 1, 103))
    b, c = po.equal_count_slices(d, 10, -2.0, 2.0)
    assert c == [11, 11, 11] + [10] * 7              # 103 = 10 * 10 + 3: the first three groups
    assert sum(c) == 103 and b[0] == -2.0 and b[-1] == 2.0
    b2, c2 = po.equal_width_slices(d, 8, -2.0, 2.0)
    assert np.allclose(np.diff(b2), 0.5) and sum(c2) == 103
    assert c2[0] == 0 and c2[-1] == 0                # the data lie in [-1, 1]


def test_affine_invariance():
    """Maps that are exact in FP64 carry the partition along: scaling by 4 and a shift by 3 of data
    on a 2^-30 grid give the same counts and the mapped boundaries."""
    d = _clusters([40, 25, 60], [0.0, 0.3, 0.9], 0.05, 5)
    d = np.round(d * 2.0 ** 30) / 2.0 ** 30
    lo, hi = d[0] - 0.5, d[-1] + 0.5
    b, c, _ = po.kmeans_slices(d, 5, lo, hi)
    for f in (lambda x: 4.0 * x, lambda x: x + 3.0):
        b2, c2, _ = po.kmeans_slices(f(d), 5, f(lo), f(hi))
        assert c2 == c
        assert np.array_equal(np.asarray(b2), f(np.asarray(b)))


def test_degenerate_inputs():
    # fewer points than groups: one point per group, K shrinks to n
    b, c, _ = po.kmeans_slices([0.1, 0.2, 0.7], 6, 0.0, 1.0)
    assert c == [1, 1, 1] and len(b) == 4
    # ties never straddle a boundary (groups are defined by value)
    d = np.sort(np.r_[np.full(7, 0.25), np.full(9, 0.5), np.linspace(0.6, 0.9, 20)])
    for K in (2, 3, 5):
        for fn in (po.equal_count_slices, lambda *a: po.kmeans_slices(*a)[:2]):
            b, c = fn(d, K, 0.0, 1.0)[:2]
            assert sum(c) == d.size
            for v, m in ((0.25, 7), (0.5, 9)):
                assert any(cnt >= m and lo <= v < hi for lo, hi, cnt in zip(b[:-1], b[1:], c))
    # a single group is the whole interval
    b, c, s = po.kmeans_slices(d, 1, 0.0, 1.0)
    assert b == [0.0, 1.0] and c == [d.size] and s == 1


def test_kmeans_keeps_tight_clusters_together():
    """Objective 1 of Section 3.1: eigenvalues closer than 1e-7 stay in one slice when the
    clusters are separated by clear gaps."""
    g = np.random.default_rng(8)
    centers = np.sort(g.uniform(0, 1, 30))
    d = np.sort(np.concatenate([c + 1e-9 * np.arange(int(g.integers(1, 6))) for c in centers]))
    b, c, _ = po.kmeans_slices(d, 6, -0.1, 1.1)
    for x in b[1:-1]:
        assert np.min(np.abs(d - x)) > 1e-7


@pytest.mark.parametrize("i0,nev,shift", [(0, 40, 0.05), (0, 25, -0.02), (30, 50, 0.01)])
def test_outer_bounds_against_closed_form_spectrum(i0, nev, shift):
    """Algorithm 4 on the 2-D Laplacian (closed-form spectrum) with 'previous' eigenvalues that
    are the current ones shifted: the bounds enclose exactly the wanted indices as counted from
    the closed form, and the number of steps is the smallest one that gets past the target."""
    m, k = 13, 11
    ab = synth.laplacian_2d_band(m, k)
    i = np.arange(1, m + 1)[:, None]
    j = np.arange(1, k + 1)[None, :]
    ev = np.sort((4 - 2 * np.cos(i * np.pi / (m + 1)) - 2 * np.cos(j * np.pi / (k + 1))).ravel())
    prev = ev - shift
    b0, bK, it_lo, it_hi, ok = po.outer_bounds(ab, prev, i0, nev, alpha=1e-3, m_hat=6)
    assert ok
    below = lambda x: int(np.sum(ev < x))
    assert below(bK) >= i0 + nev and below(b0) <= i0
    du = prev[i0 + nev - 1]
    step = max(abs(1e-3 * du), 6 * (du - prev[i0 + nev - 2]))
    target = ev[i0 + nev - 1]
    assert it_hi == max(1, int(np.floor((target - du) / step)) + 1)   # first k with du + k step > target
    dl = prev[i0]
    step2 = max(abs(1e-3 * dl), 6 * (prev[i0 + 1] - dl))
    assert (dl - it_lo * step2) <= ev[i0] and (dl - (it_lo - 1) * step2 > ev[i0] or it_lo == 1)


def test_restart_plan_invariants():
    """Start vectors after a re-slicing: unchanged slices keep their own vectors; a grown slice
    keeps every previous vector inside it and fills with random ones (mode 0) or with its nearest
    outside neighbours (mode 1); a shrunk slice keeps the ones nearest its centre."""
    g = np.random.default_rng(4)
    vals = np.sort(g.uniform(0, 1, 60))
    old_b = [0.0, 0.3, 0.6, 1.0]
    counts = [int(np.sum((vals >= lo) & (vals < hi))) for lo, hi in zip(old_b[:-1], old_b[1:])]
    plan = po.restart_plan(vals, old_b, counts)
    for (lo, hi), p in zip(zip(old_b[:-1], old_b[1:]), plan):
        assert list(p) == [k for k in range(vals.size) if lo <= vals[k] < hi]
    # a slice that grows by 5: every inside vector, then 5 random (mode 0) / 5 neighbours (mode 1)
    new_b = [0.0, 0.3, 0.6, 1.0]
    m = [counts[0] + 5, counts[1], counts[2]]
    p0 = po.restart_plan(vals, new_b, m, mode=0)[0]
    assert p0[-5:] == [-1] * 5 and all(vals[k] < 0.3 for k in p0[:-5])
    p1 = po.restart_plan(vals, new_b, m, mode=1)[0]
    nearest_above = [k for k in range(vals.size) if vals[k] >= 0.3][:5]
    assert p1[-5:] == nearest_above
    # a slice that shrinks: the kept vectors are the ones nearest the centre, in ascending order
    p = po.restart_plan(vals, [0.2, 0.5], [6])[0]
    inside = [k for k in range(vals.size) if 0.2 <= vals[k] < 0.5]
    expect = sorted(sorted(inside, key=lambda k: abs(vals[k] - 0.35))[:6])
    assert p == expect and len(inside) > 6


def test_outer_bounds_report_a_capped_search():
    """A search that runs out of counts before its target is reported, not returned as if it
    enclosed the wanted eigenvalues (Algorithm 4 with a small max_it)."""
    m, k = 13, 11
    ab = synth.laplacian_2d_band(m, k)
    i = np.arange(1, m + 1)[:, None]
    j = np.arange(1, k + 1)[None, :]
    ev = np.sort((4 - 2 * np.cos(i * np.pi / (m + 1)) - 2 * np.cos(j * np.pi / (k + 1))).ravel())
    prev = ev - 0.05                                     # every eigenvalue moved up by 0.05
    i0, nev = 30, 50
    full = po.outer_bounds(ab, prev, i0, nev, alpha=1e-3, m_hat=6)
    assert full[4] and full[3] >= 4                      # the upper search needs several counts
    capped = po.outer_bounds(ab, prev, i0, nev, alpha=1e-3, m_hat=6, max_it=3)
    assert capped[3] == 3 and not capped[4]
    assert np.sum(ev < capped[1]) < i0 + nev             # indeed not an enclosure
