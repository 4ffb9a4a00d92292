"""GPU parity of the bit-box reduction (Sec. 4.1, Alg. 1, in rounds of
pairwise disjoint boxes) against the oracle.

The whole stream (header, sequence table, packed codes), the permutation and
the decoded floats must equal the oracle's byte for byte, and every decoded
coordinate must lie within eps of its input.
"""
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


def check(pc, oracle_mod, pos, mode, eb, r, with_perm=True, autotune=False):
    omode = oracle_mod.ABS if mode == pc.PC_EB_ABS else oracle_mod.REL
    got, perm, dec = run_gpu(pc, pos, mode, eb, pc.config(r, autotune=autotune, reduce=True), with_perm)
    if autotune:  # the oracle reduces the leaves of the leaf size the autotuner chose
        r = pc.pc_stream_info(got[:96]).leaf_size
    ref, ref_perm, rounds = oracle_mod.compress_reduced(pos, omode, eb, leaf_size=r)
    assert len(got) == len(ref)
    if got != ref:
        a, b = np.frombuffer(got, np.uint8), np.frombuffer(ref, np.uint8)
        raise AssertionError(f"stream differs from the oracle at byte {int(np.flatnonzero(a != b)[0])} of {len(a)}")
    if with_perm:
        assert np.array_equal(perm, ref_perm)
    assert dec.tobytes() == oracle_mod.decompress(ref).tobytes()
    if pos.shape[0]:
        eps = pc.pc_stream_info(got[:96]).eps
        err = np.abs(pos[ref_perm].astype(np.float64) - dec.astype(np.float64))
        assert int((err > eps).sum()) == 0
    return got, rounds


CASES = [
    # generator, n, dtype, mode, eb, leaf size
    ("cosmology", 4_000, np.float32, "rel", 1e-2, 25),        # many small boxes, many rounds
    ("cosmology", 50_000, np.float32, "rel", 1e-3, 128),
    ("uniform", 65_537, np.float32, "abs", 0.5, 64),           # 1024 boxes, ragged
    ("uniform", 100_000, np.float32, "rel", 1e-4, 4096),
    ("cosmology", 1 << 18, np.float32, "rel", 1e-4, 4096),
    ("cosmology", 300_001, np.float32, "rel", 1e-3, 777),
    ("fluid", 1 << 18, np.float64, "abs", 1e-4, 4096),
    ("fluid", 100_003, np.float64, "abs", 1e-6, 1000),         # codes above 2^16 (u32 path)
    ("cosmology", 200_000, np.float64, "rel", 1e-7, 2048),     # u32 codes, float64
    ("uniform", 3_000, np.float32, "rel", 1e-3, 1),            # one particle per box
    ("uniform", 3_001, np.float32, "rel", 1e-3, 2),
    ("cosmology", 150_000, np.float32, "rel", 1e-4, 12000),    # largest leaf size
]


@pytest.mark.parametrize("gen,n,dt,mode,eb,r", CASES)
def test_reduction_matches_oracle(pc, oracle_mod, gen, n, dt, mode, eb, r):
    pos = synth.by_name(gen, n, seed=11, dtype=dt)
    m = pc.PC_EB_ABS if mode == "abs" else pc.PC_EB_REL
    got, rounds = check(pc, oracle_mod, pos, m, eb, r)
    assert rounds >= 1
    assert parse(got, with_codes=False).num_leaves <= oracle_mod.num_leaves(n, r)


def test_reduction_without_perm(pc, oracle_mod):
    pos = synth.cosmology(60_000, seed=3)
    check(pc, oracle_mod, pos, pc.PC_EB_REL, 1e-3, 256, with_perm=False)


def test_reduction_with_autotuned_leaves(pc, oracle_mod):
    pos = synth.cosmology(200_000, seed=4)
    check(pc, oracle_mod, pos, pc.PC_EB_REL, 1e-4, 4096, autotune=True)


@pytest.mark.parametrize("n", [1, 2, 3, 33, 1025])
def test_reduction_tiny(pc, oracle_mod, n):
    check(pc, oracle_mod, synth.uniform(n, seed=n), pc.PC_EB_REL, 1e-3, 16)


def test_reduction_single_leaf_is_the_plain_stream(pc, oracle_mod):
    pos = synth.cosmology(3_000, seed=5)
    got, rounds = check(pc, oracle_mod, pos, pc.PC_EB_REL, 1e-3, 4096)
    plain, _ = oracle_mod.compress(pos, oracle_mod.REL, 1e-3, leaf_size=4096)
    assert got == plain and rounds == 1


def test_reduction_identical_points(pc, oracle_mod):
    """Every code is 0: all boxes are the same point, the first takes everything."""
    pos = np.full((5_000, 3), 1.25, np.float32)
    got, rounds = check(pc, oracle_mod, pos, pc.PC_EB_ABS, 1e-3, 64)
    assert rounds == 1 and parse(got, with_codes=False).num_leaves == 1


def test_reduction_duplicated_clusters(pc, oracle_mod):
    """Copies of the same points spread over many leaves: heavy box overlap."""
    base = synth.uniform(500, seed=6, box=4.0)
    pos = np.concatenate([base] * 40)
    pos = pos[np.random.default_rng(6).permutation(len(pos))]
    check(pc, oracle_mod, pos, pc.PC_EB_ABS, 1e-2, 100)


def test_reduction_empty(pc):
    dev = torch.device("cuda:0")
    c = pc.Compressor(0, pc.PC_F32, leaf_size=pc.config(64, reduce=True), device=dev)
    size = c.compress(torch.empty((0, 3), dtype=torch.float32, device=dev), pc.PC_EB_ABS, 1e-3)
    assert size == 96


def test_reduction_more_boxes_met_than_a_batch(pc, oracle_mod):
    """625 leaves of identical points: the first box taken meets all 624 others,
    more than one search batch holds."""
    pos = np.full((40_000, 3), -3.5, np.float64)
    got, rounds = check(pc, oracle_mod, pos, pc.PC_EB_ABS, 1e-3, 64)
    assert rounds == 1 and parse(got, with_codes=False).num_leaves == 1
    base = synth.uniform(400, seed=8, box=2.0)
    pos = np.concatenate([base] * 100)
    pos = pos[np.random.default_rng(8).permutation(len(pos))]
    check(pc, oracle_mod, pos, pc.PC_EB_ABS, 5e-3, 50)
