"""The OpenMP build of the oracle (same source, -fopenmp) is the oracle: the
same streams, permutations and decoded positions as the single-threaded
build, on several threads."""
import os

import numpy as np
import pytest

import synth


@pytest.mark.parametrize("gen,n,dtype,mode,eb,r", [
    ("cosmology", 300_000, np.float32, "rel", 1e-4, 4096),
    ("uniform", 100_003, np.float32, "rel", 1e-3, 777),
    ("fluid", 120_000, np.float64, "abs", 1e-4, 2048),
    ("uniform", 5_000, np.float64, "abs", 0.5, 1),
])
def test_parallel_oracle_matches(oracle_mod, gen, n, dtype, mode, eb, r):
    os.environ.setdefault("OMP_NUM_THREADS", "4")
    pos = synth.by_name(gen, n, seed=3, dtype=dtype)
    m = oracle_mod.ABS if mode == "abs" else oracle_mod.REL
    s1, p1 = oracle_mod.compress(pos, m, eb, leaf_size=r)
    s2, p2 = oracle_mod.compress(pos, m, eb, leaf_size=r, parallel=True)
    assert s1 == s2 and np.array_equal(p1, p2)
    assert oracle_mod.decompress(s1).tobytes() == oracle_mod.decompress(s2, parallel=True).tobytes()


def test_parallel_oracle_rejects_like_the_oracle(oracle_mod):
    pos = synth.uniform(1000, seed=1)
    pos[17, 1] = np.nan
    with pytest.raises(oracle_mod.OracleError) as e:
        oracle_mod.compress(pos, oracle_mod.REL, 1e-3, parallel=True)
    assert e.value.code == oracle_mod.ERR_NONFINITE
