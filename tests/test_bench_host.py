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
