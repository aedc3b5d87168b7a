"""The benchmark's roofline arithmetic on CPU: algorithmic bytes per kernel
(every input read once, every output written once), the dominant-kernel
choice, achieved = bytes / time, and the recorded DRAM traffic, which is
used only while the kernel sources match the digest it was captured on."""
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


def test_algorithmic_bytes_per_unit_at_load_one(bench):
    n = V = q = 1 << 20
    b = bench.algo_build(4, n, V)
    assert b == {"k_hist": 4 * n, "k_partition_A": 12 * n, "k_partition_B": 16 * n, "k_binbuild": 16 * n + 4 * V}
    p = bench.algo_probe(4, n, V, q, 0.5, binned=True)
    assert p["k_hist_Q"] == 4 * q and p["k_partition_Q"] == 12 * q and p["k_unpermute"] == 12 * q
    assert p["k_probe"] == 4 * q + 4 * q + 4 * (V + 1) + 4 * n          # queries, counts, table once
    assert bench.algo_probe(4, n, V, q, 0.5, binned=True, positions=True)["k_probe"] == p["k_probe"] + 4 * q
    # 8-byte keys: (key, id) records are 12 bytes
    b8 = bench.algo_build(8, n, V)
    assert b8["k_partition_B"] == 24 * n and b8["k_binbuild"] == 24 * n + 4 * V


def test_direct_probe_counts_sectors(bench):
    q = 1 << 10
    # every query hits: offsets sector + first-key sector + the 8 sequential bytes
    assert bench.algo_probe(4, 1 << 10, 1 << 10, q, 1.0, binned=False)["k_probe"] == q * (4 + 4 + 32 + 32)


def test_roofline_picks_the_longest_kernel(bench, monkeypatch):
    monkeypatch.setattr(bench, "recorded_traffic", lambda k, u, w=None: ("traffic", k, u))
    algo = {"k_a": 1_000_000_000, "k_b": 4_000_000_000}
    prof = {"k_a": (2.0, 4), "k_b": (10.0, 2), "k_untracked": (50.0, 1)}
    roof, phases = bench.roofline(prof, algo, steps=2, elapsed_ms=100.0, hbm=1000.0, peak_src="measured",
                                  units={"k_a": 10, "k_b": 100}, workload=bench.TRAFFIC_WORKLOAD)
    assert roof["kernel"] == "k_b"                                       # the untracked kernel is not a candidate
    assert roof["achieved"] == pytest.approx(4e9 * 2 / 10e-3 / 1e9)      # 800 GB/s
    assert roof["frac"] == pytest.approx(0.8)
    assert roof["peak_nominal"] == 8000.0 and roof["frac_nominal"] == pytest.approx(0.1)  # 800 of 8000 GB/s
    assert roof["traffic"] == ("traffic", "k_b", 100.0)                  # units per launch: 100 * 2 steps / 2
    assert phases["k_a"]["avg_ms"] == 0.5 and phases["k_a"]["algo_bytes_per_launch"] == 500_000_000
    assert phases["k_untracked"]["share"] == 0.5 and "frac" not in phases["k_untracked"]


def test_recorded_traffic_follows_the_source_digest(bench, monkeypatch, tmp_path):
    csrc = tmp_path / "paper_1907_02900_gb300" / "csrc"
    csrc.mkdir(parents=True)
    (csrc / "k.cu").write_text("// v1\n")
    (tmp_path / "profiles").mkdir()
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    dig = bench.src_digest()
    (tmp_path / "profiles" / "traffic.json").write_text(json.dumps(
        {"k_probe": {"bytes_per_unit": 23.5, "units": "queries", "src_digest": dig}}))
    w = bench.TRAFFIC_WORKLOAD
    assert bench.recorded_traffic("k_probe", 1000, w) == 23500
    assert bench.recorded_traffic("k_other", 1000, w) is None
    assert bench.recorded_traffic("k_probe", 1000) is None              # another workload: no figure
    assert bench.recorded_traffic("k_probe", 1000, "join") is None
    (csrc / "k.cu").write_text("// v2\n")                               # the kernel changed since the capture
    assert bench.recorded_traffic("k_probe", 1000, w) is None


def test_committed_traffic_record_is_well_formed(bench):
    with open(os.path.join(ROOT, "profiles", "traffic.json")) as f:
        t = json.load(f)
    for k, e in t.items():
        assert e["bytes_per_unit"] > 0 and e["units"] in ("keys", "queries") and len(e["src_digest"]) == 16, k
        assert os.path.exists(os.path.join(ROOT, e["source"])), k
