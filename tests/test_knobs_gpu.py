"""The launch knobs on the GPU: threads per node (warp_node_max, the node size up
to which one warp splits a node of a level over HBM) and packing tile
(warp_leaf_max, the leaf size up to which one warp computes a leaf's bit box
and packs it).  They choose kernels, never bytes: under every setting the
stream, the permutation and the decoded floats equal the oracle's byte for
byte.  The autotuner (PC_FLAG_AUTOTUNE_KNOBS) times the settings that change a
launch on the first call of a class and keeps the fastest; the stream it
writes, and the one a plain call with its reported config writes, are the
oracle's too.
"""
import numpy as np
import pytest

import synth
from test_parity_gpu import pc, run_gpu  # noqa: F401  (pc is a fixture)

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

# gen, n, dtype, mode, eb, leaf size, flags: levels over HBM with nodes of 2^17 down to 2 r,
# and leaves packed over HBM (the leaf-size search, the reduction with the reordering)
INPUTS = [
    ("uniform", 1 << 17, np.float32, "rel", 1e-3, 256, ""),
    ("cosmology", 90_001, np.float32, "rel", 1e-4, 100, ""),
    ("fluid", 50_000, np.float64, "abs", 1e-4, 0, "autotune"),
    ("cosmology", 30_000, np.float32, "rel", 1e-3, 200, "reduce"),
]
KNOBS = [(512, 256), (1 << 16, 12000), (4096, 4096), (1, 1)]


def _oracle(oracle_mod, pos, mode, eb, r, flags):
    om = oracle_mod.ABS if mode == "abs" else oracle_mod.REL
    if flags == "reduce":
        s, p, _ = oracle_mod.compress_reduced(pos, om, eb, leaf_size=r)
        s, p, _ = oracle_mod.reorder(s, p)
        return s, p
    return oracle_mod.compress(pos, om, eb, leaf_size=r)


def _cfg(pc, r, flags, **kw):
    if flags == "autotune":
        return pc.config(r, autotune=True, **kw)
    if flags == "reduce":
        return pc.config(r, reduce=True, reorder=True, **kw)
    return pc.config(r, **kw)


@pytest.mark.parametrize("knobs", KNOBS, ids=lambda k: f"node{k[0]}-leaf{k[1]}")
@pytest.mark.parametrize("gen,n,dtype,mode,eb,r,flags", INPUTS)
def test_launch_knobs_change_no_byte(pc, oracle_mod, gen, n, dtype, mode, eb, r, flags, knobs):
    pos = synth.by_name(gen, n, seed=n % 89, dtype=dtype)
    m = pc.PC_EB_ABS if mode == "abs" else pc.PC_EB_REL
    cfg = _cfg(pc, r, flags, warp_node_max=knobs[0], warp_leaf_max=knobs[1])
    got, perm, dec = run_gpu(pc, pos, m, eb, cfg)
    r_used = pc.pc_stream_info(got[:96]).leaf_size
    ref, ref_perm = _oracle(oracle_mod, pos, mode, eb, r_used, flags)
    assert got == ref
    assert np.array_equal(perm, ref_perm)
    assert dec.tobytes() == oracle_mod.decompress(ref).tobytes()


@pytest.mark.parametrize("gen,n,dtype,mode,eb,r,flags", INPUTS)
def test_knob_autotuner_reports_a_config_a_plain_call_reproduces(pc, oracle_mod, gen, n, dtype, mode, eb, r, flags):
    pos = synth.by_name(gen, n, seed=n % 83, dtype=dtype)
    m = pc.PC_EB_ABS if mode == "abs" else pc.PC_EB_REL
    dt = pc.PC_F32 if dtype == np.float32 else pc.PC_F64
    pc.autotune_reset()
    cfg = _cfg(pc, r, flags, tune_knobs=True)
    before, tuned = pc.tuned_config(n, dt, cfg)
    assert not tuned and before.warp_node_max == pc.PC_DEFAULT_WARP_NODE_MAX
    first, perm1, _ = run_gpu(pc, pos, m, eb, cfg)  # tunes the class
    chosen, tuned = pc.tuned_config(n, dt, cfg)
    assert tuned
    assert chosen.flags == cfg.flags & ~pc.PC_FLAG_AUTOTUNE_KNOBS and chosen.leaf_size == cfg.leaf_size
    assert chosen.warp_node_max in (512, 1024, 2048, 4096, 8192)
    assert chosen.warp_leaf_max in (256, 512, 1024, 2048, 4096)
    again, perm2, _ = run_gpu(pc, pos, m, eb, cfg)  # the tuned class
    plain, perm3, dec = run_gpu(pc, pos, m, eb, chosen)
    r_used = pc.pc_stream_info(first[:96]).leaf_size
    ref, ref_perm = _oracle(oracle_mod, pos, mode, eb, r_used, flags)
    assert first == ref and again == ref and plain == ref
    for p in (perm1, perm2, perm3):
        assert np.array_equal(p, ref_perm)
    assert dec.tobytes() == oracle_mod.decompress(ref).tobytes()
    # a class of its own: another bit length of n is untuned
    _, other = pc.tuned_config(4 * n, dt, cfg)
    assert not other


def test_knob_autotuner_in_a_batch(pc, oracle_mod):
    """Batch items carrying PC_FLAG_AUTOTUNE_KNOBS tune their classes inside the
    lanes (several items share a class, one tunes it while the others run with
    the defaults); every item's stream is still its plain call's."""
    dev = torch.device("cuda:0")
    pc.autotune_reset()
    rng = np.random.default_rng(5)
    pos_list, ebs = [], []
    for k in range(12):
        n = int(rng.integers(20_000, 70_000))
        pos_list.append(synth.by_name("cosmology" if k % 2 else "uniform", n, seed=k, dtype=np.float32))
        ebs.append(1e-3 if k % 3 else 1e-4)
    cfg = pc.config(256, tune_knobs=True)
    dpos = [torch.from_numpy(p).to(dev) for p in pos_list]
    outs = [torch.empty(pc.pc_compress_bound(p.shape[0], pc.PC_F32, cfg), dtype=torch.uint8, device=dev)
            for p in pos_list]
    sizes, statuses = pc.pc_compress_batch([(p, pc.PC_EB_REL, eb, cfg) for p, eb in zip(dpos, ebs)], outs, lanes=4)
    torch.cuda.synchronize()
    assert all(st == pc.PC_OK for st in statuses)
    for pos, eb, o, size in zip(pos_list, ebs, outs, sizes):
        ref, _ = oracle_mod.compress(pos, oracle_mod.REL, eb, leaf_size=256, want_perm=False)
        assert o[:size].cpu().numpy().tobytes() == ref


def test_noalloc_uses_tuned_knobs_without_tuning(pc, oracle_mod):
    """The entry point that allocates nothing never tunes (a class it meets
    untuned stays untuned) and writes the plain stream either way."""
    dev = torch.device("cuda:0")
    pc.autotune_reset()
    pos = synth.by_name("uniform", 50_000, seed=3, dtype=np.float32)
    cfg = pc.config(256, tune_knobs=True)
    out = torch.empty(pc.pc_compress_bound(pos.shape[0], pc.PC_F32, cfg), dtype=torch.uint8, device=dev)
    size = pc.pc_compress_noalloc(torch.from_numpy(pos).to(dev), pc.PC_EB_REL, 1e-3, out, leaf_size=cfg)
    torch.cuda.synchronize()
    _, tuned = pc.tuned_config(pos.shape[0], pc.PC_F32, cfg)
    assert not tuned
    ref, _ = oracle_mod.compress(pos, oracle_mod.REL, 1e-3, leaf_size=256, want_perm=False)
    assert out[:size].cpu().numpy().tobytes() == ref
