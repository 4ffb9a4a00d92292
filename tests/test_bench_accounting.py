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


def test_batch_workload_config_is_sized_like_the_leaf_autotuner_alone():
    """The batch-256 line runs both autotuners (leaf size and launch knobs); the
    knob flag changes no size the library reports for it (host-only queries)."""
    import paper_2404_02826_gb300 as pc
    from paper_2404_02826_gb300 import build as pcbuild

    pcbuild.build()
    pc.load()
    cfg = bench.BATCH_CFG(pc)
    assert cfg.flags == pc.PC_FLAG_AUTOTUNE_LEAF | pc.PC_FLAG_AUTOTUNE_KNOBS
    assert (cfg.leaf_size, cfg.warp_node_max, cfg.warp_leaf_max) == (0, 0, 0)
    items = [(12_345, pc.PC_F32), (2_000_000, pc.PC_F64), (9_999_999, pc.PC_F32)]
    for n, dt in items:
        assert pc.pc_compress_bound(n, dt, cfg) == pc.pc_compress_bound(n, dt, pc.LEAF_AUTO)
        assert pc.pc_compress_workspace_size(n, dt, cfg) == pc.pc_compress_workspace_size(n, dt, pc.LEAF_AUTO)
    assert pc.pc_compress_batch_workspace_size([(n, dt, cfg) for n, dt in items], 16) == \
        pc.pc_compress_batch_workspace_size([(n, dt, pc.LEAF_AUTO) for n, dt in items], 16)


def test_knob_summary_counts_the_tuned_classes():
    """The batch line's `tuned_knobs`: how many classes the launch-knob autotuner
    tuned and how often it picked each value (here from imported classes)."""
    import paper_2404_02826_gb300 as pc
    from paper_2404_02826_gb300 import build as pcbuild

    pcbuild.build()
    pc.load()
    pc.autotune_reset()
    assert bench.knob_summary(pc) == {"classes": 0, "warp_node_max": {}, "warp_leaf_max": {}}
    mk = lambda bits, node, leaf: {"n_bits": bits, "dtype": 0, "device": 0, "flags": 1, "leaf_size": 0,
                                   "warp_node_max": node, "warp_leaf_max": leaf}
    pc.autotune_import([mk(15, 2048, 1024), mk(16, 4096, 1024), mk(17, 4096, 512)])
    assert bench.knob_summary(pc) == {"classes": 3, "warp_node_max": {"2048": 1, "4096": 2},
                                      "warp_leaf_max": {"512": 1, "1024": 2}}
    pc.autotune_reset()
