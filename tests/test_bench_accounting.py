"""bench.py's roofline accounting on CPU: the algorithmic bytes per launch it
divides by a kernel's time, and the DRAM traffic it takes from the committed
ncu captures only while their kernels' sources are unchanged."""
import json
import os
import shutil
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def test_algorithmic_bytes_per_kernel():
    n, esz, cb, s = 1 << 20, 4, 2, 123_456
    ab = bench.algorithmic_bytes
    # the scatter reads and writes all three code arrays (and the input index with a permutation)
    assert ab("k_scatter", n, esz, cb, s) == 12 * n
    assert ab("k_scatter", n, esz, cb, s, with_idx=True) == 20 * n
    # quantize: positions in, codes out; range: positions in
    assert ab("k_quantize", n, esz, cb, s) == 12 * n + 6 * n
    assert ab("k_range", n, 8, cb, s) == 24 * n
    # one digit pass of the select reads the split axis only
    assert ab("k_hist", n, esz, cb, s) == 2 * n and ab("k_count", n, esz, 4, s) == 4 * n
    # the subtree reads the codes once and writes the stream; the decoder reads the stream and
    # writes the positions; the search pass only reads
    assert ab("k_subtree", n, esz, cb, s) == 6 * n + s
    assert ab("k_decode", n, esz, cb, s) == s + 12 * n
    assert ab("k_subtree_cost", n, esz, cb, s) == 6 * n
    # the reduction's take kernel: the whole reduction's bytes spread over its launches
    assert ab("k_rd_take", n, esz, cb, s, launches=4) == (6 + 8) * n / 4
    assert ab("k_unknown", n, esz, cb, s) is None


def test_traffic_only_for_unchanged_sources(tmp_path, monkeypatch):
    with open(os.path.join(ROOT, "profiles", "dram_traffic.json")) as f:
        rec = json.load(f)["k_scatter"]
    if rec["source_hash"] != bench.source_hash(rec["sources"]):
        pytest.skip("the committed capture predates the current k_scatter sources")
    n = 1 << 27
    assert bench.measured_traffic("k_scatter", "cosmology-2^27-f32-rel1e-4", n) == pytest.approx(
        rec["dram_bytes_per_particle"] * n)
    # the same tree with one of the kernel's sources changed: no traffic figure
    for rel in ["profiles/dram_traffic.json"] + rec["sources"]:
        os.makedirs(os.path.dirname(tmp_path / rel), exist_ok=True)
        shutil.copy(os.path.join(ROOT, rel), tmp_path / rel)
    with open(tmp_path / rec["sources"][0], "a") as f:
        f.write("\n// changed\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.measured_traffic("k_scatter", "cosmology-2^27-f32-rel1e-4", n) is None
    assert bench.measured_traffic("k_nothing", "cosmology-2^27-f32-rel1e-4", n) is None
