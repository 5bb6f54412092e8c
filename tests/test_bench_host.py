"""bench.py's host-side arithmetic (CPU only): the algorithmic-byte model of the roofline,
the reached-edge count behind GTEPS, the traffic scaling from the small ncu capture, the
argument parser and the reference arm's metric table."""
import numpy as np

import bench


def test_reached_edges_and_algo_bytes(gg, orc):
    # a path 0 -> 1 -> 2 plus an unreachable vertex 3 with two out-edges
    g = gg.from_edges(4, [0, 1, 3, 3], [1, 2, 0, 2], [5, 5, 1, 1])
    d = orc.dijkstra(g, 0)
    m_r, n_r = bench.reached_edges(g, d)
    assert (m_r, n_r) == (2, 3)  # edges out of 0 and 1 (2 has none); 0, 1, 2 reached
    assert bench.algo_bytes(m_r, n_r, g.n) == 12 * 2 + 28 * 3 + 4 * 4


def test_algo_bytes_of_the_road_workload_per_source():
    # the road-like 4900 x 4900 workload's figure quoted with the roofline: 12 m + 28 n + 4 n
    # bytes per source when every vertex is reached (the road graph is one component)
    n, m = 23997150, 82565692
    per_source = bench.algo_bytes(m, n, n)
    assert per_source == 12 * m + 32 * n
    assert per_source * 8 == 14069576832  # the bench's bytes_per_launch for 8 sources


def test_scaled_traffic_follows_vertices_times_sources(monkeypatch):
    cap = dict(bench.TRAFFIC_CAPTURE)
    monkeypatch.setattr(bench, "kernel_sha", lambda: cap["kernel_sha"])
    full = bench.scaled_traffic("road", cap["n"] * 4, cap["sources"], 1)
    assert full == int(cap["bytes"] * 4)
    half = bench.scaled_traffic("road", cap["n"], cap["sources"] // 2, 1)
    assert half == int(cap["bytes"] / 2)
    # another graph kind, the barrier-free engine or a changed kernel: no figure
    assert bench.scaled_traffic("rmat", cap["n"], cap["sources"], 1) is None
    assert bench.scaled_traffic("road", cap["n"], cap["sources"], 2) is None
    monkeypatch.setattr(bench, "kernel_sha", lambda: "0" * 16)
    assert bench.scaled_traffic("road", cap["n"], cap["sources"], 1) is None


def test_rmat_traffic_only_for_the_captured_launch(monkeypatch):
    """The full-size R-MAT capture is reported only for the launch it measured: the same
    workload, scale, sources, hot-first order, schedule and kernel code."""
    cap = bench.RMAT_TRAFFIC
    monkeypatch.setattr(bench, "kernel_sha", lambda: cap["kernel_sha"])
    sched = cap["rmat-sssp"]["schedule"]
    assert bench.rmat_traffic("rmat-sssp", 24, 8, True, sched) == cap["rmat-sssp"]["bytes"]
    assert bench.rmat_traffic("rmat-wbfs", 24, 8, True, cap["rmat-wbfs"]["schedule"]) == \
        cap["rmat-wbfs"]["bytes"]
    assert bench.rmat_traffic("rmat-wbfs", 24, 8, True, (2, 1024, 512, 4096)) is None
    assert bench.rmat_traffic("rmat-sssp", 24, 8, True, (128,) + tuple(sched[1:])) is None
    assert bench.rmat_traffic("rmat-sssp", 22, 8, True, sched) is None
    assert bench.rmat_traffic("rmat-sssp", 24, 2, True, sched) is None
    assert bench.rmat_traffic("rmat-sssp", 24, 8, False, sched) is None
    assert bench.rmat_traffic("road-sssp", 24, 8, True, sched) is None
    monkeypatch.setattr(bench, "kernel_sha", lambda: "0" * 16)
    assert bench.rmat_traffic("rmat-sssp", 24, 8, True, sched) is None


def test_kernel_sha_covers_the_kernel_sources():
    sha = bench.kernel_sha()
    assert len(sha) == 16 and int(sha, 16) >= 0
    assert any(f.endswith("og_kernels.cu") for f in bench.KERNEL_SOURCES)


def test_parser_defaults_and_workloads():
    a = bench.parse_args([])
    assert (a.gpus, a.workload, a.warmup) == (1, "road-sssp", 3) and a.warmup >= 3
    assert a.impl == "ours" and a.side == 4900 and a.sources == 8
    for w in ("rmat-wbfs", "rmat-sssp", "batch", "serve", "road-bf", "road-lazy",
              "rmat-lazy", "rmat-kcore", "rmat-setcover"):
        assert bench.parse_args(["--workload", w]).workload == w


def test_reference_metrics_name_every_workload():
    choices = {"road-sssp", "rmat-wbfs", "rmat-sssp", "batch", "serve", "road-bf",
               "road-lazy", "rmat-lazy", "rmat-kcore", "rmat-setcover"}
    assert set(bench.REF_METRIC) == choices
    assert "queries/s" in bench.REF_METRIC["batch"] and "GTEPS" in bench.REF_METRIC["road-sssp"]


def test_reference_arm_prints_one_contract_line_on_rank_zero(monkeypatch, capsys):
    import json
    monkeypatch.setenv("RANK", "0")
    monkeypatch.setenv("WORLD_SIZE", "1")
    bench.run_reference(bench.parse_args(["--impl", "reference", "--side", "48",
                                          "--sources", "2", "--steps", "3", "--warmup", "1"]))
    lines = [ln for ln in capsys.readouterr().out.splitlines() if ln.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["metric"] == bench.REF_METRIC["road-sssp"]
    assert d["unit"] == "GTEPS" and d["value"] > 0 and d["higher_is_better"] is True
    assert (d["steps"], d["warmup"], d["n_gpus"]) == (3, 1, 1)
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] == 1 and cb["value"] == d["value"]
    assert d["e2e"] == {"value": d["value"], "unit": "GTEPS", "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}


def test_reference_arm_is_silent_on_other_ranks(monkeypatch, capsys):
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    bench.run_reference(bench.parse_args(["--impl", "reference", "--side", "48"]))
    assert capsys.readouterr().out == ""


def test_clock_summary_takes_loaded_samples_and_active_reasons():
    na = "Not Active"
    rows = [
        f"0, 1980, 2070, 150.2, 0x0000000000000000, {na}, {na}, {na}, {na}",  # idle
        f"0, 2070, 2070, 910.5, 0x0000000000000000, {na}, {na}, {na}, {na}",
        f"0, 2055, 2070, 1390.0, 0x0000000000000004, {na}, {na}, {na}, Active",
        f"0, 2040, 2070, 1201.7, 0x0000000000000004, {na}, {na}, {na}, Active",
        "0, [N/A], 2070, [N/A], [N/A], [N/A], [N/A], [N/A], [N/A]",  # unreadable sample
        "",
    ]
    s = bench.clock_summary(rows)
    assert s["samples"] == 4 and s["sm_max_mhz"] == 2070
    assert s["sm_mhz"] == 2055  # median of the three samples above 200 W
    assert s["reasons"] == ["sw_power_cap"] and s["power_w_max"] == 1390.0
    slow = rows[1].replace(f"{na}, {na}, {na}, {na}", f"Active, {na}, Active, {na}")
    assert bench.clock_summary([slow])["reasons"] == ["hw_slowdown", "sw_thermal_slowdown"]
    # no load at all: the median of every sample; nothing parsed: marked unsampled
    assert bench.clock_summary(rows[:1])["sm_mhz"] == 1980
    assert bench.clock_summary([])["reasons"] == ["unsampled"]
