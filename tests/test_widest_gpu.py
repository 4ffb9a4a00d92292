"""GPU parity of the widest-cell split axis (PC_FLAG_WIDEST_AXIS; Sec. 4.1 leaves
the axis open) against the oracle's second tree rule: whole stream,
permutation and decoded floats byte for byte, every coordinate within eps."""
import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pc():
    import paper_2404_02826_gb300 as pc
    from paper_2404_02826_gb300 import build as b

    b.build()
    pc.load()
    assert torch.cuda.is_available()
    return pc


def check(pc, oracle_mod, pos, mode, eb, r, reduce=False, reorder=False):
    dev = torch.device("cuda:0")
    dpos = torch.from_numpy(np.ascontiguousarray(pos)).to(dev)
    dtype = pc.PC_F32 if pos.dtype == np.float32 else pc.PC_F64
    c = pc.Compressor(pos.shape[0], dtype, leaf_size=pc.config(r, reduce=reduce, reorder=reorder, widest=True),
                      with_perm=True, device=dev)
    size = c.compress(dpos, mode, eb)
    got = c.out[:size].cpu().numpy().tobytes()
    out = torch.empty_like(dpos)
    if pos.shape[0]:
        c.decompress(c.out, out, size)
    torch.cuda.synchronize()
    perm = c.perm[: pos.shape[0]].cpu().numpy().astype(np.int64)
    om = oracle_mod.ABS if mode == pc.PC_EB_ABS else oracle_mod.REL
    if reduce:
        ref, rperm, _ = oracle_mod.compress_reduced(pos, om, eb, leaf_size=r, widest=True)
    else:
        ref, rperm = oracle_mod.compress(pos, om, eb, leaf_size=r, widest=True)
    if reorder:
        ref, rperm, _ = oracle_mod.reorder(ref, rperm)
    assert len(got) == len(ref)
    if got != ref:
        a, b = np.frombuffer(got, np.uint8), np.frombuffer(ref, np.uint8)
        raise AssertionError(f"stream differs from the oracle at byte {int(np.flatnonzero(a != b)[0])} of {len(a)}")
    assert np.array_equal(perm, rperm)
    dec = out.cpu().numpy()
    assert dec.tobytes() == oracle_mod.decompress(ref).tobytes()
    if pos.shape[0]:
        eps = pc.pc_stream_info(got[:96]).eps
        assert np.abs(pos[rperm].astype(np.float64) - dec.astype(np.float64)).max() <= eps
    return got


CASES = [
    # generator, n, dtype, mode, eb, leaf size
    ("fluid", 1 << 18, np.float64, "abs", 1e-4, 4096),          # a 1 x 0.5 x 0.59 box: x is cut more often
    ("fluid", 100_003, np.float64, "abs", 1e-6, 1000),          # u32 codes
    ("cosmology", 1 << 18, np.float32, "rel", 1e-4, 64),        # deep: tiled levels, warp medians, warp nodes
    ("cosmology", 300_001, np.float32, "rel", 1e-3, 777),
    ("uniform", 1 << 20, np.float32, "rel", 1e-3, 4096),
    ("uniform", 40_000, np.float32, "rel", 1e-3, 1),
]


@pytest.mark.parametrize("gen,n,dt,mode,eb,r", CASES)
def test_widest_matches_oracle(pc, oracle_mod, gen, n, dt, mode, eb, r):
    pos = synth.by_name(gen, n, seed=31, dtype=dt)
    check(pc, oracle_mod, pos, pc.PC_EB_ABS if mode == "abs" else pc.PC_EB_REL, eb, r)


def test_widest_slab_differs_from_depth_rule(pc, oracle_mod):
    rng = np.random.default_rng(4)
    pos = (rng.random((200_000, 3)) * np.array([64.0, 8.0, 1.0])).astype(np.float32)
    got = check(pc, oracle_mod, pos, pc.PC_EB_ABS, 0.01, 2048)
    plain, _ = oracle_mod.compress(pos, oracle_mod.ABS, 0.01, leaf_size=2048)
    assert got != plain and len(got) < len(plain)


def test_widest_with_reduction_and_reordering(pc, oracle_mod):
    pos = synth.fluid(60_000, seed=32)
    check(pc, oracle_mod, pos, pc.PC_EB_ABS, 1e-4, 512, reduce=True, reorder=True)
    check(pc, oracle_mod, synth.cosmology(80_000, seed=33), pc.PC_EB_REL, 1e-3, 1000, reorder=True)


@pytest.mark.parametrize("n", [1, 2, 3, 33])
def test_widest_tiny(pc, oracle_mod, n):
    check(pc, oracle_mod, synth.uniform(n, seed=n), pc.PC_EB_REL, 1e-3, 1)
