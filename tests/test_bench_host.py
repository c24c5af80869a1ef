"""Host-side logic of bench.py: query subsets, the oracle sample, the clock
summary (throttle reasons decide whether a run is kept), and the traffic
records keyed by kernel source hashes."""
import json
import os

import numpy as np
import pytest

import bench


def test_parse_query_list():
    assert bench.parse_query_list("3,5,8", 10) == [3, 5, 8]
    assert bench.parse_query_list("2:5", 10) == [2, 3, 4]
    assert bench.parse_query_list(":3", 10) == [0, 1, 2]
    assert bench.parse_query_list("7:", 9) == [7, 8]
    assert bench.parse_query_list("0:100", 4) == [0, 1, 2, 3]


def test_cpu_sample_is_deterministic_and_bounded():
    class Q:
        def __init__(self, b):
            self.bound = b
    qs = [Q(b) for b in (1e9, 5.0, 3e7, 1e3, 2e7, 1.0, 9e9, 10.0, 11.0, 12.0, 13.0, 14.0)]
    idx = bench.cpu_sample(qs)
    assert idx == [1, 3, 4, 5, 7, 8, 9, 10]
    assert all(qs[i].bound <= 2e7 for i in idx)


def test_clock_summary_reasons():
    ok = "0, 2070, 2070, 900.1 W, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active"
    capped = "0, 1980, 2070, 1399.9 W, 0x0000000000000004, Not Active, Not Active, Not Active, Active"
    hot = "0, 1500 MHz, 2070 MHz, 1200 W, 0x40, Not Active, Active, Not Active, Not Active"
    s = bench.summarize_clocks([ok, ok, capped])
    assert s["sm_mhz"] == 2070 and s["sm_max_mhz"] == 2070 and s["reasons"] == ["sw_power_cap"] and s["samples"] == 3
    s = bench.summarize_clocks([ok, hot, "garbage", "0, [N/A], [N/A], x, y, a, b, c, d"])
    assert s["reasons"] == ["hw_thermal_slowdown"] and s["samples"] == 2
    assert bench.summarize_clocks([]) is None


def test_traffic_records(tmp_path, monkeypatch):
    os.makedirs(tmp_path / "profiles")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "kernel_source_hash", lambda k: "abc")
    path = tmp_path / "profiles" / "k_query_medium_traffic.json"
    assert bench.recorded_traffic("k_query", "medium", 100.0) == (None, None)        # no record
    json.dump({"kernel_source_sha": "abc", "same_workload": True, "dram_bytes_per_launch": 42.0,
               "ratio_to_alg_bytes": 0.5, "source": "s"}, open(path, "w"))
    assert bench.recorded_traffic("k_query", "medium", 100.0) == (42.0, "s")        # measured on this workload
    json.dump({"kernel_source_sha": "abc", "same_workload": False, "ratio_to_alg_bytes": 0.5, "source": "r"},
              open(path, "w"))
    assert bench.recorded_traffic("k_query", "medium", 100.0) == (50.0, "r")        # scaled by algorithmic bytes
    json.dump({"kernel_source_sha": "old", "same_workload": True, "dram_bytes_per_launch": 42.0}, open(path, "w"))
    assert bench.recorded_traffic("k_query", "medium", 100.0) == (None, None)        # kernel changed since


@pytest.mark.parametrize("kernel,workload", [("k_query", "medium"), ("k_batch", "batched")])
def test_committed_traffic_records_are_well_formed(kernel, workload):
    rec = json.load(open(os.path.join(bench.ROOT, "profiles", f"{kernel}_{workload}_traffic.json")))
    assert rec["kernel"] == kernel and rec["workload"] == workload
    assert rec["dram_bytes_per_launch"] > 0 and rec["ratio_to_alg_bytes"] > 0
    assert rec["command"].startswith("ncu ") and "--clock-control none" in rec["command"]


def test_cpu_baseline_reports_cores_and_one_thread():
    import synth
    g = synth.workload_graph("tiny")
    qs = synth.queries("tiny")
    for q in qs:
        q.bound = 1.0                                        # every tiny query is in the sample
    out = bench.cpu_baseline(qs, g)
    assert out["kind"] == "oracle" and out["cores"] >= 1 and out["value"] > 0
    assert out["one_thread"]["value"] > 0 and out["one_thread"]["query"] in range(len(qs))


def test_cpu_baseline_edge_mode_counts_edge_matches():
    """With edge=True the baseline counts the oracle's edge-isomorphic matches."""
    import oracle
    import synth
    g = synth.workload_graph("tiny")
    qs = synth.queries("tiny")
    for q in qs:
        q.bound = 1.0
    out = bench.cpu_baseline(qs, g, edge=True)
    assert out["unit"] == "edge matches/s" and out["value"] > 0
    O = oracle.OracleGraph.from_synth(g)
    total = sum(oracle.count_edge(O, q)[0] for q in qs)
    assert f"{total} edge matches" in out["sample"]


def test_edge_workload_recipe():
    """The edge workload's graph has bounded degree (its line graph stays
    within the transform's 2^31-edge limit) and its queries are connected
    walks with at least one edge."""
    import synth
    w = synth.WORKLOADS["edge"]
    assert w.graph.kind == "er" and w.graph.n == 1 << 20 and w.graph.m == 4_000_000
    assert bench.data_desc("edge") == "synthetic (seeded Erdos-Renyi graph, random-walk queries)"
    assert bench.data_desc("medium") == "synthetic (seeded R-MAT graph, random-walk queries)"
    g = synth.workload_graph("edge")
    deg = np.bincount(np.concatenate([g.src, g.dst]), minlength=g.n).astype(np.int64)
    assert int((deg * (deg - 1) // 2).sum()) < 2 ** 31
    qs = synth.queries("edge", 4)
    assert all(1 <= len(q.src) <= 32 and w.k_lo <= q.k <= w.k_hi for q in qs)
