"""Host logic of bench.py that needs no GPU: the kernel-source digest that
ties the committed ncu traffic to the code it was captured from, and the
algorithmic byte models behind the roofline figures."""
import json
import os
import shutil
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


@pytest.fixture
def tree(tmp_path, monkeypatch):
    """A copy of the kernel sources and profiles under a scratch root."""
    csrc = tmp_path / "paper_2110_00511_gb300" / "csrc"
    csrc.mkdir(parents=True)
    for f in bench.KERNEL_SOURCES:
        shutil.copy(os.path.join(ROOT, "paper_2110_00511_gb300", "csrc", f), csrc / f)
    shutil.copytree(os.path.join(ROOT, "profiles"), tmp_path / "profiles")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    return tmp_path


def _edit(path, old, new):
    text = path.read_text()
    assert old in text
    path.write_text(text.replace(old, new, 1))


def test_digest_ignores_comments_and_whitespace(tree):
    before = bench.source_digest()
    f = tree / "paper_2110_00511_gb300" / "csrc" / "ash_kernels.cuh"
    _edit(f, "#pragma once", "// an added comment line\n/* and a block\n   comment */   #pragma once")
    assert bench.source_digest() == before


def test_digest_follows_code_changes(tree):
    before = bench.source_digest()
    f = tree / "paper_2110_00511_gb300" / "csrc" / "ash_device.cuh"
    _edit(f, "constexpr uint32_t kFpBit = 0x80000000u;", "constexpr uint32_t kFpBit = 0x40000000u;")
    assert bench.source_digest() != before


def test_traffic_reported_only_for_the_captured_code(tree):
    data = json.load(open(tree / "profiles" / "traffic.json"))
    data["source_digest"] = bench.source_digest()
    (tree / "profiles" / "traffic.json").write_text(json.dumps(data))
    want = data["kernels"]["insert_claim"]["dram_bytes_per_launch_full_size"]
    assert bench.measured_traffic("insert_claim") == want
    assert bench.measured_traffic("no_such_kernel") is None
    f = tree / "paper_2110_00511_gb300" / "csrc" / "ash_dim.cu"
    f.write_text(f.read_text() + "\nnamespace ash { int changed_code = 1; }\n")
    assert bench.measured_traffic("insert_claim") is None


def test_byte_models_per_unit():
    """The per-unit figures of the byte-model table for d = 3 (key stride 4)."""
    assert bench.bytes_find(1, 0) == 81 and bench.bytes_find(0, 1) == 49
    assert bench.bytes_claim(1) == 80
    # commit: 9 per key + one winner bit per key; a winner adds its key row
    # (12), kB row (16), slot rewrite (32) and value row read + write
    n, win, vb = 8000, 5000, 4
    base = n * 9 + n // 8
    assert bench.bytes_commit(n, win, vb) == base + win * (12 + 16 + 32 + 2 * vb)
    assert bench.bytes_commit(n, win, vb, heap_identity=False) - bench.bytes_commit(n, win, vb) == 4 * win
    # listing: the identity heap writes only the live indices
    assert bench.bytes_list(1000, 600) == 4 * 600
    assert bench.bytes_list(1000, 600, heap_identity=False) == 4 * 400 + 3 * 125 + 4 * 600
    assert bench.bytes_gather_keys(10) == 10 * (4 + 16 + 12)
    assert bench.bytes_erase(3, 2) == bench.bytes_find(3, 2) + 3 * 36


def _full_result():
    """A result dict shaped like the GPU arm's, with every side block filled
    (sweep, per-op, batched, serving over five rates, TSDF, per-kernel)."""
    point = {"n": 100_000_000, "rho": 0.5, "unique": 50_000_000, "working_set_x_l2": 36.3, "ranged": True,
             "activate": {"ms": 7.1, "keys_per_s": 1.4e10, "algo_gbs": 1680.3, "frac_hbm": 0.2461,
                          "speedup_vs_input_order": 1.1123,
                          "input_order": {"ms": 7.9, "keys_per_s": 1.27e10, "frac_hbm": 0.2251,
                                          "frac_random_access_roofline": 0.61234}},
             "find": {"ms": 4.1, "keys_per_s": 2.43e10, "algo_gbs": 1970.1, "frac_hbm": 0.2937,
                      "frac_random_access_roofline": 0.7912}}
    rate = {m: {"p50_ms": 1.234567, "p99_ms": 7.654321, "p999_ms": 9.87, "req_per_s": 9512.25,
                "keys_per_s": 1.3e9, "avg_requests_per_batch": 1.7, "growth_rehashes": 3}
            for m in ("served", "served_pinned_dma", "served_zero_copy", "sequential_plain")}
    kern = {f"k{i}": {"traced_launches": 5, "ms_per_launch": 0.0123456, "share": 0.1, "algo_bytes_per_launch": 1e8,
                      "achieved_gbs": 3111.2, "frac": 0.4634} for i in range(12)}
    return {
        "metric": bench.METRIC, "value": 24312345678.9, "unit": bench.UNIT, "n_gpus": 1, "steps": 20, "warmup": 5,
        "ms_per_step": 0.32912345, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "int32", "data": "synthetic",
        "config": {"workload": bench.WORKLOAD, "points": 4_000_000, "voxel_m": 0.005, "key_dim": 3,
                   "unique_voxels": 3847013, "value": "int32 point index", "step": "x" * 300,
                   "l2": "flushed (256 MiB write) between steps",
                   "parallelism": "single GPU"},
        "gpu_launches": 240,
        "roofline": {"bound": "hbm", "kernel": "insert_claim", "achieved": 3110.123, "peak": 6794.5,
                     "peak_kind": "measured (MEASURED_PEAKS.json hbm_gbs, copy bandwidth)", "unit": "GB/s",
                     "frac": 0.4577, "traffic": 202700000},
        "cpu_baseline": {"value": 2.5e6, "unit": bench.UNIT, "cores": 1, "kind": "oracle", "sample": "y" * 60,
                         "all_cores": {"value": 2.9e7, "unit": bench.UNIT, "cores": 16, "kind": "oracle",
                                       "sample": "z" * 60},
                         "tsdf_frame": {"ms_per_frame": 7100.0}},
        "e2e": {"value": 1.33e10, "unit": bench.UNIT, "h2d_bytes_per_step": 48_000_000,
                "d2h_bytes_per_step": 64_000_008, "path": "p" * 200, "steps": 20,
                "zero_copy": {"value": 8.8e9, "path": "q" * 200}},
        "graph_step": {"ms_median": 0.302, "value": 2.65e10, "note": "n" * 200},
        "clocks": {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": [], "samples": 8,
                   "samples_in_timed_region": True, "interval_ms": 50},
        "kernels": kern, "random_access_roofline": {f"p{i}": 1.0 for i in range(20)},
        "sweep": {"l2_bytes": 132_120_576, "points": [dict(point, n=10 ** (4 + i // 3)) for i in range(12)] + [point]},
        "ops": {"insert": {"ms": 1.0}}, "batched": {
            "batched_graph": {"ms_median": 1.2, "ms_p99": 1.4, "ops_per_s": 1.5e10},
            "plain_per_map": {"ms_median": 7.2, "ms_p99": 8.4, "ops_per_s": 2.5e9}, "maps": 64},
        "serving": {"default_mode": "served_pinned_dma",
                    "rates": {str(r): dict(rate, offered_keys_per_s=1e9) for r in (2000, 5000, 10000, 20000, 50000)}},
        "tsdf": {"ms_per_frame": 0.49, "kernels": kern}, "tsdf_block_map": {"kernels": kern},
        "source_digest": "0123456789abcdef",
    }


def test_summary_line_is_short_and_carries_the_contract(tmp_path, capsys):
    """The one stdout line stays well under what a tail capture keeps, parses
    as JSON, and holds the contract's keys; the full result goes to the
    detail file."""
    full = _full_result()
    assert len(json.dumps(full)) > 8000
    detail = tmp_path / "detail.json"
    bench.emit(full, str(detail))
    out = capsys.readouterr().out.strip().splitlines()
    assert len(out) == 1
    line = out[-1]
    assert len(line.encode()) <= bench.COMPACT_LIMIT
    d = json.loads(line)
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config", "gpu_launches", "roofline", "cpu_baseline",
              "e2e", "clocks"):
        assert k in d, k
    assert d["value"] > 0 and d["steps"] == 20 and d["warmup"] == 5
    for k in ("bound", "achieved", "peak", "unit", "frac", "traffic"):
        assert k in d["roofline"]
    assert d["cpu_baseline"]["cores"] == 1 and d["cpu_baseline"]["all_cores"]["cores"] == 16
    assert d["e2e"]["h2d_bytes_per_step"] > 0 and d["e2e"]["d2h_bytes_per_step"] > 0
    assert d["config"]["workload"] == bench.WORKLOAD
    assert "served" in d["highlights"] and "sweep" in d["highlights"] and "batched_G" in d["highlights"]
    # a ranged point reports its own rate and copy-peak fraction, and the
    # input-order calls' roofline fraction and rate beside them
    act = d["highlights"]["sweep"]["act"]
    assert act[1] == pytest.approx(0.2461, abs=1e-3) and act[2] == pytest.approx(0.6123, abs=1e-3)
    assert act[3] == pytest.approx(12.7, abs=0.1)
    assert json.load(open(detail)) == full


def test_summary_line_reference_arm(capsys):
    line = {"impl": "reference", "metric": bench.METRIC, "value": 9.4e6, "unit": bench.UNIT, "n_gpus": 1,
            "steps": 20, "warmup": 5, "ms_per_step": 850.0, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "int32", "data": "synthetic",
            "config": {"workload": bench.WORKLOAD, "points": 4_000_000, "voxel_m": 0.005},
            "cpu_baseline": {"value": 9.4e6, "unit": bench.UNIT, "cores": 16, "kind": "oracle", "sample": "s"},
            "e2e": {"value": 9.4e6, "unit": bench.UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    bench.emit(line, None)
    d = json.loads(capsys.readouterr().out.strip().splitlines()[-1])
    assert d["impl"] == "reference" and d["cpu_baseline"]["cores"] == 16 and d["e2e"]["value"] == 9.4e6


def test_all_cores_oracle_step_counts_every_point():
    """The sharded oracle pass covers every point exactly once (each key
    lands in one shard) and reports insert + find keys."""
    from concurrent.futures import ThreadPoolExecutor
    import numpy as np
    rng = np.random.default_rng(0)
    pts = rng.uniform(-1, 1, size=(5000, 3)).astype(np.float32)
    with ThreadPoolExecutor(max_workers=3) as pool:
        assert bench.oracle_all_cores_step(pts, 0.05, pool, 3) == 2 * len(pts)
    keys = rng.integers(-100, 100, size=(1000, 3)).astype(np.int32)
    own = bench._owner(keys, 4)
    assert own.min() >= 0 and own.max() < 4
    assert np.array_equal(own, bench._owner(keys.copy(), 4))


def test_random_and_streamed_split_adds_up():
    """The (random, streamed) splits add up to the algorithmic byte models,
    and the random-access fraction is 1 exactly when the measured time equals
    the probe time for the random part plus the copy time for the rest."""
    r, s_ = bench.split_find(700, 300)
    assert r + s_ == bench.bytes_find(700, 300)
    assert r == 32 * 1000 + 32 * 700
    r, s_ = bench.split_activate(1000, 600)
    assert r + s_ == bench.bytes_claim(1000) + bench.bytes_commit(1000, 600, 0)
    assert r == 64 * 1000 + 32 * 600
    ms = (3.2e9 / 40e9 + 1.0e9 / 6000e9) * 1000
    f = bench.random_access_fraction(ms, 3.2e9, 1.0e9, 40.0, 6000.0)
    assert abs(f - 1.0) < 1e-12
    assert bench.random_access_fraction(2 * ms, 3.2e9, 1.0e9, 40.0, 6000.0) == pytest.approx(0.5)
    assert bench.random_access_fraction(ms, 1, 1, None, 6000.0) is None
