"""CPU-only checks of the C-ABI library: it builds, loads without a GPU, exports
every entry point that include/pc.h declares, and its host-only calls (sizes,
header parsing, status strings) agree with the oracle's streams."""
import os
import re

import numpy as np
import pytest

import synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="session")
def pc():
    from paper_2404_02826_gb300 import build as b

    b.build()
    import paper_2404_02826_gb300 as pc

    pc.load()
    return pc


def declared_functions():
    names = []
    for h in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if not h.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", h)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names += re.findall(r"^\s*(?:const\s+)?[A-Za-z_][\w\s\*]*?\b(pc_\w+)\s*\(", text, flags=re.M)
    return sorted(set(names))


def test_every_declared_symbol_is_exported(pc):
    lib = pc.load()
    names = declared_functions()
    assert len(names) >= 12
    for name in names:
        assert hasattr(lib, name), name
    assert set(names) == set(pc.EXPORTS)


def test_status_strings(pc):
    for code in range(0, 9):
        s = pc.pc_error_string(code)
        assert isinstance(s, str) and s
    assert pc.pc_format_version() == 1


@pytest.mark.parametrize("gen,n,r", [("uniform", 5000, 300), ("cosmology", 20000, 4096), ("fluid", 9000, 64),
                                     ("uniform", 1, 4096), ("uniform", 0, 4096)])
def test_stream_info_and_bound_match_oracle_streams(pc, oracle_mod, gen, n, r):
    pos = synth.by_name(gen, n, seed=2) if n else np.zeros((0, 3), np.float32)
    stream, _ = oracle_mod.compress(pos, oracle_mod.REL, 1e-3, leaf_size=r)
    info = pc.pc_stream_info(stream[:96])
    n0, dt, nl, nw = oracle_mod.stream_header(stream)
    assert (info.n, info.dtype, info.num_leaves, info.payload_words) == (n0, dt, nl, nw)
    assert info.total_bytes == len(stream)
    assert info.leaf_size == r
    dtype = pc.PC_F32 if pos.dtype == np.float32 else pc.PC_F64
    assert pc.pc_compress_bound(n, dtype, r) >= len(stream)
    assert nl == oracle_mod.num_leaves(n, r)


def test_leaf_count_rule_matches_oracle(pc, oracle_mod):
    # the library sizes its leaf table from (n, r) alone; the bound exposes it
    rng = np.random.default_rng(0)
    for _ in range(300):
        n = int(rng.integers(0, 1 << 22))
        r = int(rng.integers(1, 12001))
        L = oracle_mod.num_leaves(n, r)
        # at most 3 M bits per particle: lossless axes store M-bit coordinates (Sec. 4.1)
        b = pc.pc_compress_bound(n, pc.PC_F32, r)
        assert b == 96 + 36 * L + 4 * ((96 * n + 31) // 32)
        b = pc.pc_compress_bound(n, pc.PC_F64, r)
        assert b == 96 + 36 * L + 4 * ((192 * n + 31) // 32)


def test_argument_errors_without_gpu(pc):
    with pytest.raises(pc.PCError) as e:
        pc.pc_compress_bound(10, 7)
    assert e.value.status == pc.PC_ERR_ARG
    with pytest.raises(pc.PCError):
        pc.pc_compress_workspace_size(10, pc.PC_F32, leaf_size=pc.PC_MAX_LEAF_SIZE + 1)
    with pytest.raises(pc.PCError) as e:
        pc.pc_stream_info(b"XXXX" + bytes(92))
    assert e.value.status == pc.PC_ERR_CORRUPT
    with pytest.raises(pc.PCError):
        pc.pc_compress_bound(1 << 31, pc.PC_F32)


def test_autotune_flag_sizes_and_rejections(pc):
    """Autotuning sizes the stream bound and the workspace for its smallest
    candidate (PC_AUTOTUNE_MIN_LEAF); unknown flag bits and maxima below 16 are
    rejected."""
    n = 1_000_000
    auto = pc.pc_compress_bound(n, pc.PC_F32, pc.LEAF_AUTO)
    assert auto == pc.pc_compress_bound(n, pc.PC_F32, pc.PC_AUTOTUNE_MIN_LEAF)
    assert pc.pc_compress_workspace_size(n, pc.PC_F32, pc.LEAF_AUTO) >= pc.pc_compress_workspace_size(n, pc.PC_F32)
    assert pc.pc_compress_bound(n, pc.PC_F32, -512) == pc.pc_compress_bound(n, pc.PC_F32, pc.PC_AUTOTUNE_MIN_LEAF)
    cfg = pc.pc_config(0, 32)  # no such flag
    out = pc.ctypes.c_uint64()
    assert pc.load().pc_compress_bound(n, pc.PC_F32, pc.ctypes.byref(cfg), pc.ctypes.byref(out)) == pc.PC_ERR_ARG
    # the bit-box reduction writes no more sequences than leaves, and needs more scratch
    red = pc.config(0, reduce=True)
    assert pc.pc_compress_bound(n, pc.PC_F32, red) == pc.pc_compress_bound(n, pc.PC_F32)
    assert pc.pc_compress_workspace_size(n, pc.PC_F32, red) > pc.pc_compress_workspace_size(n, pc.PC_F32)
    both = pc.config(0, autotune=True, reduce=True)
    assert pc.pc_compress_bound(n, pc.PC_F32, both) == auto
    # reordering keeps the stream size and needs its own scratch
    ro = pc.config(0, reorder=True)
    assert pc.pc_compress_bound(n, pc.PC_F32, ro) == pc.pc_compress_bound(n, pc.PC_F32)
    assert pc.pc_compress_workspace_size(n, pc.PC_F32, ro) > pc.pc_compress_workspace_size(n, pc.PC_F32)
    with pytest.raises(pc.PCError) as e:
        pc.pc_compress_bound(n, pc.PC_F32, -8)
    assert e.value.status == pc.PC_ERR_ARG


def test_launch_knobs_sizes_rejections_and_tuned_config(pc):
    """The launch knobs (threads per node, packing tile) change neither the stream
    bound nor the workspace; values above their maxima are rejected; the tuned
    config of a class nobody has compressed is the call's own config, without
    PC_FLAG_AUTOTUNE_KNOBS and with the defaults filled in (no device needed)."""
    n = 300_000
    L = pc.load()
    out = pc.ctypes.c_uint64()
    base_bound = pc.pc_compress_bound(n, pc.PC_F32, 512)
    base_ws = pc.pc_compress_workspace_size(n, pc.PC_F32, 512)
    for knobs in ((1, 1), (512, 256), (pc.PC_MAX_WARP_NODE_MAX, pc.PC_MAX_LEAF_SIZE)):
        cfg = pc.config(512, warp_node_max=knobs[0], warp_leaf_max=knobs[1])
        assert pc.pc_compress_bound(n, pc.PC_F32, cfg) == base_bound
        assert pc.pc_compress_workspace_size(n, pc.PC_F32, cfg) == base_ws
    tuned_cfg = pc.config(512, tune_knobs=True)
    assert pc.pc_compress_bound(n, pc.PC_F32, tuned_cfg) == base_bound
    assert pc.pc_compress_workspace_size(n, pc.PC_F32, tuned_cfg) == base_ws
    for bad in (pc.config(512, warp_node_max=pc.PC_MAX_WARP_NODE_MAX + 1),
                pc.config(512, warp_leaf_max=pc.PC_MAX_LEAF_SIZE + 1)):
        assert L.pc_compress_bound(n, pc.PC_F32, pc.ctypes.byref(bad), pc.ctypes.byref(out)) == pc.PC_ERR_ARG
    pc.autotune_reset()
    got, tuned = pc.tuned_config(n, pc.PC_F32, pc.config(512, reduce=True, tune_knobs=True))
    assert not tuned
    assert (got.leaf_size, got.flags) == (512, pc.PC_FLAG_BOX_REDUCTION)
    assert (got.warp_node_max, got.warp_leaf_max) == (pc.PC_DEFAULT_WARP_NODE_MAX, pc.PC_DEFAULT_WARP_LEAF_MAX)
    got, _ = pc.tuned_config(n, pc.PC_F32, pc.config(512, tune_knobs=True, warp_node_max=700, warp_leaf_max=90))
    assert (got.warp_node_max, got.warp_leaf_max) == (700, 90)
    # the query wants the flag, and checks the config like the compression does
    plain = pc.config(512)
    tuned_out = pc.pc_config()
    flag = pc.ctypes.c_int()
    assert L.pc_tuned_config(n, pc.PC_F32, pc.ctypes.byref(plain), pc.ctypes.byref(tuned_out),
                             pc.ctypes.byref(flag)) == pc.PC_ERR_ARG
    bad = pc.config(512, tune_knobs=True, warp_leaf_max=pc.PC_MAX_LEAF_SIZE + 1)
    assert L.pc_tuned_config(n, pc.PC_F32, pc.ctypes.byref(bad), pc.ctypes.byref(tuned_out),
                             pc.ctypes.byref(flag)) == pc.PC_ERR_ARG


def _tuned(n_bits, dtype, flags, leaf, node, leaf_max, device=0):
    return {"n_bits": n_bits, "dtype": dtype, "device": device, "flags": flags, "leaf_size": leaf,
            "warp_node_max": node, "warp_leaf_max": leaf_max}


def _key(c):
    return tuple(sorted(c.items()))


def test_tuned_classes_export_import_and_json(pc, tmp_path):
    """Tuned launch-knob classes go out and come back (the autotuner's persisted
    cache): imported classes are what pc_tuned_config reports for calls of those
    classes, an import replaces a class's entry, a JSON file written by
    autotune_save restores the same table, and bad entries are refused whole."""
    pc.autotune_reset()
    assert pc.autotune_export() == []
    a = _tuned(17, pc.PC_F32, pc.PC_FLAG_AUTOTUNE_LEAF, 0, 4096, 512)
    b = _tuned(20, pc.PC_F64, 0, 256, 1024, 2048)
    c = _tuned(24, pc.PC_F32, pc.PC_FLAG_BOX_REDUCTION | pc.PC_FLAG_REORDER, 4096, 8192, 256)
    pc.autotune_import([a, b, c])
    assert sorted(map(_key, pc.autotune_export())) == sorted(map(_key, [a, b, c]))
    got, tuned = pc.tuned_config(100_000, pc.PC_F32, pc.config(0, autotune=True, tune_knobs=True))  # 17 bits
    assert tuned and (got.warp_node_max, got.warp_leaf_max) == (4096, 512)
    assert got.flags == pc.PC_FLAG_AUTOTUNE_LEAF and got.leaf_size == 0
    got, tuned = pc.tuned_config(600_000, pc.PC_F64, pc.config(256, tune_knobs=True))  # 20 bits
    assert tuned and (got.warp_node_max, got.warp_leaf_max) == (1024, 2048)
    # another leaf size, bit length or dtype is another class
    assert not pc.tuned_config(600_000, pc.PC_F64, pc.config(512, tune_knobs=True))[1]
    assert not pc.tuned_config(1_100_000, pc.PC_F64, pc.config(256, tune_knobs=True))[1]
    assert not pc.tuned_config(600_000, pc.PC_F32, pc.config(256, tune_knobs=True))[1]
    # re-importing a class replaces its knobs; duplicates within one import keep the last
    b2 = dict(b, warp_node_max=512)
    pc.autotune_import([b, b2])
    table = {(_key(dict(x, warp_node_max=0, warp_leaf_max=0))): x for x in pc.autotune_export()}
    assert len(table) == 3 and table[_key(dict(b, warp_node_max=0, warp_leaf_max=0))]["warp_node_max"] == 512
    # JSON round trip
    path = tmp_path / "knobs.json"
    assert pc.autotune_save(path) == 3
    before = sorted(map(_key, pc.autotune_export()))
    pc.autotune_reset()
    assert pc.autotune_load(path) == 3
    assert sorted(map(_key, pc.autotune_export())) == before
    # bad entries: nothing of the import is entered
    L = pc.load()
    for bad in (dict(a, n_bits=32), dict(a, dtype=2), dict(a, device=256), dict(a, device=-1),
                dict(a, flags=pc.PC_FLAG_AUTOTUNE_KNOBS), dict(a, flags=64), dict(a, warp_node_max=0),
                dict(a, warp_leaf_max=0), dict(a, warp_node_max=pc.PC_MAX_WARP_NODE_MAX + 1),
                dict(a, warp_leaf_max=pc.PC_MAX_LEAF_SIZE + 1), dict(a, flags=0, leaf_size=pc.PC_MAX_LEAF_SIZE + 1),
                dict(a, leaf_size=8)):  # the leaf-size search needs a largest candidate of at least 16
        arr = (pc.pc_tuned_class * 2)()
        for i, entry in enumerate((_tuned(5, pc.PC_F32, 0, 0, 2048, 1024), bad)):
            for f, v in entry.items():
                setattr(arr[i], f, v)
        assert L.pc_autotune_import(arr, 2) == pc.PC_ERR_ARG, bad
        assert sorted(map(_key, pc.autotune_export())) == before
    arr = (pc.pc_tuned_class * 1)()
    arr[0].n_bits, arr[0].warp_node_max, arr[0].warp_leaf_max, arr[0].reserved = 5, 2048, 1024, 1
    assert L.pc_autotune_import(arr, 1) == pc.PC_ERR_ARG
    with open(tmp_path / "other.json", "w") as f:
        f.write('{"format": "something-else", "version": 1, "classes": []}')
    with pytest.raises(ValueError):
        pc.autotune_load(tmp_path / "other.json")
    pc.autotune_reset()


def test_tuned_class_table_capacity(pc):
    """The table holds 256 classes; an import that needs more room than is free
    enters nothing."""
    pc.autotune_reset()
    full = [_tuned(bits, dt, 0, leaf, 2048, 1024) for bits in range(32) for dt in (0, 1) for leaf in (0, 1, 2, 3)]
    assert len(full) == 256
    pc.autotune_import(full)
    assert len(pc.autotune_export()) == 256
    pc.autotune_import(full[:10])  # the same classes again: no room needed
    with pytest.raises(pc.PCError) as e:
        pc.autotune_import([_tuned(5, 0, 0, 7, 2048, 1024)])
    assert e.value.status == pc.PC_ERR_CAPACITY
    pc.autotune_reset()
    with pytest.raises(pc.PCError) as e:
        pc.autotune_import(full + [_tuned(5, 0, 0, 7, 2048, 1024)])
    assert e.value.status == pc.PC_ERR_CAPACITY
    assert pc.autotune_export() == []
