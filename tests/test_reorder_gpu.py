"""GPU parity of the reordering for the entropy coder (Sec. 4.2, after Fig. 4)
against the oracle: the oracle compresses (plain or with the bit-box
reduction) and reorders; the CUDA path must write the same bytes and the same
permutation, and decode within eps."""
import numpy as np
import pytest

import synth
from streamfmt import parse

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


def run_gpu(pc, pos, mode, eb, cfg, with_perm=True):
    dev = torch.device("cuda:0")
    dpos = torch.from_numpy(np.ascontiguousarray(pos)).to(dev)
    dtype = pc.PC_F32 if pos.dtype == np.float32 else pc.PC_F64
    c = pc.Compressor(pos.shape[0], dtype, leaf_size=cfg, with_perm=with_perm, device=dev)
    size = c.compress(dpos, mode, eb)
    stream = c.out[:size].clone()
    out = torch.empty_like(dpos)
    if pos.shape[0]:
        c.decompress(stream, out, size)
    torch.cuda.synchronize()
    perm = c.perm[: pos.shape[0]].cpu().numpy().astype(np.int64) if with_perm else None
    return stream.cpu().numpy().tobytes(), perm, out.cpu().numpy()


def check(pc, oracle_mod, pos, mode, eb, r, reduce=False, autotune=False, with_perm=True):
    omode = oracle_mod.ABS if mode == pc.PC_EB_ABS else oracle_mod.REL
    got, perm, dec = run_gpu(pc, pos, mode, eb, pc.config(r, autotune=autotune, reduce=reduce, reorder=True),
                             with_perm)
    if autotune:
        r = pc.pc_stream_info(got[:96]).leaf_size
    if reduce:
        base, bperm, _ = oracle_mod.compress_reduced(pos, omode, eb, leaf_size=r)
    else:
        base, bperm = oracle_mod.compress(pos, omode, eb, leaf_size=r)
    ref, ref_perm, _ = oracle_mod.reorder(base, bperm)
    assert len(got) == len(ref) == len(base)
    if got != ref:
        a, b = np.frombuffer(got, np.uint8), np.frombuffer(ref, np.uint8)
        raise AssertionError(f"stream differs from the oracle at byte {int(np.flatnonzero(a != b)[0])} of {len(a)}")
    if with_perm:
        assert np.array_equal(perm, ref_perm)
    assert dec.tobytes() == oracle_mod.decompress(ref).tobytes()
    if pos.shape[0]:
        eps = pc.pc_stream_info(got[:96]).eps
        assert np.abs(pos[ref_perm].astype(np.float64) - dec.astype(np.float64)).max() <= eps
    return got


CASES = [
    # generator, n, dtype, mode, eb, leaf size, reduce
    ("cosmology", 1 << 18, np.float32, "rel", 1e-4, 4096, False),
    ("cosmology", 300_001, np.float32, "rel", 1e-3, 777, False),
    ("fluid", 1 << 18, np.float64, "abs", 1e-4, 4096, False),
    ("fluid", 100_003, np.float64, "abs", 1e-6, 1000, False),       # u32 codes
    ("cosmology", 200_000, np.float64, "rel", 1e-7, 2048, False),   # u32 codes, wide R-indices
    ("uniform", 40_000, np.float32, "rel", 1e-3, 1, False),         # one particle per sequence
    ("cosmology", 150_000, np.float32, "rel", 1e-4, 12000, False),  # 8-byte keys of sequences above 8192
    ("uniform", 24_000, np.float64, "rel", 1e-8, 12000, False),     # 16-byte keys above 8192: global memory
    ("cosmology", 50_000, np.float32, "rel", 1e-3, 128, True),
    ("fluid", 1 << 18, np.float64, "abs", 1e-4, 4096, True),
    ("uniform", 65_537, np.float32, "abs", 0.5, 64, True),
]


@pytest.mark.parametrize("gen,n,dt,mode,eb,r,reduce", CASES)
def test_reorder_matches_oracle(pc, oracle_mod, gen, n, dt, mode, eb, r, reduce):
    pos = synth.by_name(gen, n, seed=21, dtype=dt)
    check(pc, oracle_mod, pos, pc.PC_EB_ABS if mode == "abs" else pc.PC_EB_REL, eb, r, reduce=reduce)


def test_reorder_without_perm_and_autotuned(pc, oracle_mod):
    pos = synth.cosmology(120_000, seed=22)
    check(pc, oracle_mod, pos, pc.PC_EB_REL, 1e-4, 4096, with_perm=False)
    check(pc, oracle_mod, pos, pc.PC_EB_REL, 1e-4, 4096, autotune=True)


@pytest.mark.parametrize("n", [1, 2, 3, 33])
def test_reorder_tiny(pc, oracle_mod, n):
    check(pc, oracle_mod, synth.uniform(n, seed=n), pc.PC_EB_REL, 1e-3, 16)


def test_reorder_one_long_sequence(pc, oracle_mod):
    """The reduction merges 625 leaves of identical points into one sequence of
    40000 particles: sorted in global memory."""
    got = check(pc, oracle_mod, np.full((40_000, 3), 2.0, np.float32), pc.PC_EB_ABS, 1e-3, 64, reduce=True)
    assert parse(got, with_codes=False).num_leaves == 1
    base = synth.uniform(400, seed=23, box=2.0)
    pos = np.concatenate([base] * 100)
    pos = pos[np.random.default_rng(23).permutation(len(pos))]
    check(pc, oracle_mod, pos, pc.PC_EB_ABS, 5e-3, 50, reduce=True)
