"""Re-slicing from the previous eigenvalues (Section 3.1: Algorithm 3, Approach-1, Approach-2):
the library's host implementation against the oracle, bit for bit (boundaries and counts),
and the argument checks of the C ABI.  No GPU needed."""
import numpy as np
import pytest

from oracle import partition_oracle as po


@pytest.fixture(scope="module")
def pk():
    from paper_2012_00506_gb300 import build
    build.build()
    import paper_2012_00506_gb300 as pk
    pk.load()
    return pk


def _cases():
    g = np.random.default_rng(17)
    out = []
    out.append(("uniform", np.sort(g.uniform(-1, 1, 1638)), 8))
    cl = np.concatenate([c + 0.01 * g.standard_normal(s) for c, s in
                         zip([0.0, 1.0, 2.5, 3.0, 4.2], [30, 50, 20, 40, 70])])
    out.append(("clusters", np.sort(cl), 5))
    out.append(("clusters, more slices", np.sort(cl), 13))
    mix = np.concatenate([g.normal(m, s, int(k)) for m, s, k in
                          zip(g.uniform(-1, 1, 6), g.uniform(0.01, 0.2, 6), g.integers(20, 400, 6))])
    out.append(("mixture", np.sort(mix), 64))
    ties = np.sort(np.r_[np.full(7, 0.25), np.full(9, 0.5), np.linspace(0.6, 0.9, 20)])
    out.append(("ties", ties, 5))
    out.append(("fewer points than slices", np.array([0.1, 0.2, 0.7]), 6))
    out.append(("one slice", np.sort(g.uniform(0, 1, 50)), 1))
    return out


@pytest.mark.parametrize("name,d,K", _cases(), ids=[c[0] for c in _cases()])
def test_library_partitions_match_oracle(pk, name, d, K):
    b0, bK = float(d[0] - 0.1), float(d[-1] + 0.1)
    b, c, sw = pk.partition(d, K, b0, bK, method=pk.PART_KMEANS)
    ob, oc, osw = po.kmeans_slices(d, K, b0, bK)
    assert np.array_equal(b, np.asarray(ob)) and list(c) == oc and sw == osw
    assert int(c.sum()) == d.size
    b, c, _ = pk.partition(d, K, b0, bK, method=pk.PART_EQUAL_COUNT)
    ob, oc = po.equal_count_slices(d, K, b0, bK)
    assert np.array_equal(b, np.asarray(ob)) and list(c) == oc
    b, c, _ = pk.partition(d, K, b0, bK, method=pk.PART_EQUAL_WIDTH)
    ob, oc = po.equal_width_slices(d, K, b0, bK)
    assert np.array_equal(b, np.asarray(ob)) and list(c) == oc


def test_kmeans_sweep_cap_and_arguments(pk):
    g = np.random.default_rng(3)
    d = np.sort(np.concatenate([c + 0.05 * g.standard_normal(60) for c in (0.0, 0.4, 0.7, 2.0)]))
    b, c, sw = pk.partition(d, 4, -1.0, 3.0, max_sweeps=1)
    ob, oc, osw = po.kmeans_slices(d, 4, -1.0, 3.0, max_sweeps=1)
    assert sw == osw == 1 and np.array_equal(b, np.asarray(ob)) and list(c) == oc
    lib = pk.load()
    x = np.ascontiguousarray(d)
    out_b = np.zeros(5)
    out_c = np.zeros(4, dtype=np.int32)
    k = np.zeros(1, dtype=np.int32)
    args = lambda method=0, n=x.size, K=4, b0=-1.0, bK=3.0, ms=10, data=x: lib.pdeshep_partition(
        method, n, data.ctypes.data, K, b0, bK, ms, out_b.ctypes.data, out_c.ctypes.data, k.ctypes.data, None)
    assert args() == 0
    assert args(method=3) == -1
    assert args(n=0) == -2
    assert args(data=np.ascontiguousarray(x[::-1])) == -3       # not ascending
    assert args(K=0) == -4
    assert args(b0=float(x[0]) + 1e-9) == -5
    assert args(bK=float(x[-1])) == -6                         # the last point must lie below bK
    assert args(ms=0) == -7


@pytest.mark.parametrize("mode", [0, 1])
def test_restart_plan_matches_oracle(pk, mode):
    g = np.random.default_rng(12 + mode)
    vals = g.uniform(-1, 1, 300)                  # previous Ritz values, column order
    vals[50:55] = 0.125                            # ties
    bounds = np.sort(np.r_[-1.2, g.uniform(-1, 1, 6), 1.2])
    m0 = g.integers(0, 90, bounds.size - 1).astype(np.int32)
    plan = pk.restart_plan(vals, bounds, m0, mode)
    oplan = po.restart_plan(vals, list(bounds), list(m0), mode)
    assert [list(p) for p in plan] == oplan
    lib = pk.load()
    src = np.zeros(int(m0.sum()), dtype=np.int64)
    assert lib.pdeshep_restart_plan(vals.size, vals.ctypes.data, m0.size, bounds[::-1].copy().ctypes.data,
                                    m0.ctypes.data, mode, src.ctypes.data) == -4   # bounds not ascending
    assert lib.pdeshep_restart_plan(vals.size, vals.ctypes.data, m0.size, bounds.ctypes.data, m0.ctypes.data, 2,
                                    src.ctypes.data) == -6


def test_randomized_parity(pk):
    """300 random inputs (uniform, many ties, tight clusters, growing gaps; K from 1 to 19, also
    above n): boundaries, counts and sweeps identical to the oracle for all three methods."""
    g = np.random.default_rng(0)
    for trial in range(300):
        n = int(g.integers(1, 60))
        kind = trial % 4
        if kind == 0:
            d = g.uniform(-1, 1, n)
        elif kind == 1:
            d = np.round(g.uniform(0, 1, n) * 5) / 5
        elif kind == 2:
            d = np.concatenate([c + 1e-9 * g.standard_normal(int(g.integers(1, 5)))
                                for c in g.uniform(0, 3, max(1, n // 3))])
        else:
            d = np.cumsum(g.exponential(1.0, n)) ** 2
        d = np.sort(d)
        K = int(g.integers(1, 20))
        b0, bK = float(d[0] - g.uniform(0.01, 1)), float(d[-1] + g.uniform(0.01, 1))
        b, c, sw = pk.partition(d, K, b0, bK, method=pk.PART_KMEANS)
        ob, oc, osw = po.kmeans_slices(d, K, b0, bK)
        assert np.array_equal(b, np.asarray(ob)) and list(c) == oc and sw == osw
        b, c, _ = pk.partition(d, K, b0, bK, method=pk.PART_EQUAL_COUNT)
        ob, oc = po.equal_count_slices(d, K, b0, bK)
        assert np.array_equal(b, np.asarray(ob)) and list(c) == oc
