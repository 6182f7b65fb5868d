"""Host-side logic of bench.py on the CPU: which roofline a kernel group is measured against, the
dominant group, the traffic lookup keyed by the sources' hash, and the SCF partition targets."""
import importlib.util
import json
import os

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def bench():
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def _peaks():
    return {"fp32_tflops": 76.6, "fp64_tflops": 1.06, "bf16_tflops_sustained": 1741.4, "bf16_source": "test"}


def test_solve_group_roofline_follows_the_autotuned_solve(bench):
    tb = bench.group_bounds(_peaks())
    assert tb["solve"][0] == "alu" and tb["solve"][1] == 76.6
    tc = bench.solve_bound(tb, {"rhs_chunk": 128, "rhs_chunk_early": 256})
    assert tc["solve"][0] == "tensor"
    assert tc["solve"][1] == pytest.approx(bench.BF16_SUSTAINED_TFLOPS / 6)  # bf16x6 products
    simt = bench.solve_bound(tb, {"rhs_chunk": 32, "rhs_chunk_early": 0})
    assert simt["solve"] == tb["solve"]
    assert tb["factor"] == tc["factor"]  # only the solve group changes


def test_roofline_picks_the_largest_critical_path_group(bench):
    tb = bench.group_bounds(_peaks())
    groups = {g: 0.0 for g in ("inertia", "factor", "solve", "accum", "gemm", "small", "bandmm", "eig")}
    ms = dict(groups, inertia=5000.0, solve=1600.0, factor=470.0, gemm=300.0)
    fl = dict(groups, solve=68.0e12 * 1.6, factor=4.4e12, gemm=4.2e12)
    meas = {"kg_ms": ms, "kg_fl": fl, "kg_n": {g: 1 for g in groups}, "t_s": 2.9,
            "tuned": {"rhs_chunk": 256, "rhs_chunk_early": 256}}
    roof, table = bench.roofline(meas, tb, "no-such-workload")
    assert roof["kernel_group"] == "solve"  # the side-stream inertia group is never the headline
    assert roof["bound"] == "tensor"
    assert roof["achieved"] == pytest.approx(68.0, rel=1e-3)
    assert roof["frac"] == pytest.approx(68.0 / (bench.BF16_SUSTAINED_TFLOPS / 6), rel=1e-3)
    assert roof["traffic"] is None
    assert table["factor"]["tflops"] == pytest.approx(4.4e12 / 0.47 / 1e12, rel=1e-3)


def test_traffic_is_reported_only_for_the_captured_sources(bench, tmp_path, monkeypatch):
    h = bench.source_hash("solve")
    assert h and len(h) == 12
    prof = tmp_path / "profiles"
    prof.mkdir()
    (prof / "traffic.json").write_text(json.dumps(
        {"wl": {"solve": {"source_hash": h, "dram_bytes_per_launch": 123},
                "factor": {"source_hash": "000000000000", "dram_bytes_per_launch": 456}}}))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "source_hash", lambda g: h if g == "solve" else "ffffffffffff")
    assert bench.traffic_for("solve", "wl") == 123
    assert bench.traffic_for("factor", "wl") is None   # the kernel changed since the capture
    assert bench.traffic_for("solve", "other") is None


def test_solve_hash_covers_every_solve_source(bench):
    files = bench.GROUP_SOURCES["solve"]
    assert set(files) >= {"band_lu.cu", "solve_tc.cu", "solve_tm.cu"}


def test_partition_targets_and_m0_rule(bench):
    c5 = bench.CONFIGS["c5"]
    ks = c5.targets()
    assert ks[0] == 0 and ks[-1] == c5.nev and len(ks) == c5.nslices + 1
    assert all(0 <= ks[i + 1] - ks[i] - c5.nev // c5.nslices <= 1 for i in range(c5.nslices))
    for m in (1, 10, 33, 34, 100, 153, 154):
        m0 = bench.m0_rule(m)
        assert m0 >= 1.3 * m - 1e-9 and m0 >= m + 10 and (m0 == m + 10 or m0 - 1 < 1.3 * m)
