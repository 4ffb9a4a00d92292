"""The leaf-size autotuner on the GPU against the rule it states: descend from
the largest candidate leaves while the stream shrinks, and keep the last depth
before it grows (candidates: depths d with ceil(n / 2^d) between
min(PC_AUTOTUNE_MIN_LEAF, max) and the maximum).  The oracle gives the stream
size at every candidate depth; the GPU must choose the same depth and write the
oracle's stream at that leaf size byte for byte.  The cases cover a search that
runs on the levels over HBM and one costed on chip, windows of candidates that
start below the on-chip pass's root depth, u32 codes, the permutation and the
widest-cell split axis.
"""
import numpy as np
import pytest

import synth
from test_parity_gpu import pc, run_gpu  # noqa: F401  (pc is a fixture)

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

CASES = [
    # gen, n, dtype, mode, eb, largest candidate (0: PC_MAX_LEAF_SIZE), widest, with_perm
    ("cosmology", 300_000, np.float32, "rel", 1e-4, 0, False, True),
    ("cosmology", 250_000, np.float32, "rel", 1e-3, 1024, False, False),
    ("uniform", 120_000, np.float32, "rel", 1e-2, 0, False, True),
    ("fluid", 200_000, np.float64, "abs", 1e-4, 0, False, False),
    ("fluid", 180_000, np.float64, "abs", 1e-6, 0, False, True),
    ("cosmology", 200_000, np.float32, "rel", 1e-4, 0, True, True),
    ("uniform", 40_000, np.float32, "rel", 1e-3, 8000, False, False),
    ("cosmology", 70_001, np.float32, "rel", 5e-4, 300, False, True),
    # 2^20 u16 codes, no permutation: the on-chip pass at depth 5 costs depths 6-11, the stream
    # still shrinks there (r = 128 wins), so the search resumes over HBM from the pass's
    # arrangement and its depth-10 node records
    ("cosmology", 1 << 20, np.float32, "rel", 1e-4, 0, False, False),
]


@pytest.mark.parametrize("gen,n,dtype,mode,eb,r_hi,widest,with_perm", CASES)
def test_autotune_keeps_the_last_depth_before_the_stream_grows(pc, oracle_mod, gen, n, dtype, mode, eb, r_hi,
                                                               widest, with_perm):
    pos = synth.by_name(gen, n, seed=n % 97, dtype=dtype)
    m = pc.PC_EB_ABS if mode == "abs" else pc.PC_EB_REL
    om = oracle_mod.ABS if mode == "abs" else oracle_mod.REL
    got, perm, dec = run_gpu(pc, pos, m, eb, pc.config(r_hi, autotune=True, widest=widest), with_perm=with_perm)
    r = pc.pc_stream_info(got[:96]).leaf_size

    hi = r_hi or pc.PC_MAX_LEAF_SIZE
    lo = min(pc.PC_AUTOTUNE_MIN_LEAF, hi)
    ceil_at = lambda d: -(-n // (1 << d))
    first = next(d for d in range(64) if ceil_at(d) <= hi)
    cands = [first] + [d for d in range(first + 1, 64) if ceil_at(d) >= lo]
    sizes = {d: len(oracle_mod.compress(pos, om, eb, leaf_size=ceil_at(d), want_perm=False, widest=widest)[0])
             for d in cands}
    expect = next(d for d in cands if d + 1 not in sizes or sizes[d + 1] >= sizes[d])
    assert r == ceil_at(expect), (r, ceil_at(expect), sizes)

    ref, ref_perm = oracle_mod.compress(pos, om, eb, leaf_size=r, widest=widest)
    assert got == ref
    if with_perm:
        assert np.array_equal(perm, ref_perm)
    assert dec.tobytes() == oracle_mod.decompress(ref).tobytes()
