"""Randomized properties of the oracle on tiny inputs (hypothesis; CPU only).

Each drawn input (size, generator, scale, bound mode, leaf size, duplicated
points) must give: every decoded coordinate within eps (Sec. 3); every input
index exactly once in the permutation; leaves of floor/ceil sizes of the
median rule, none above r (Sec. 4.1); every code within [0, 2^m - 2] (Eq. 1);
decoded codes equal to the quantized input; payload bits equal to the sum over
leaves of (sum m_d)(count - 1) (Sec. 4.2, the storage term); and the reduced
and reordered streams keep every particle and the bound.
"""
import numpy as np
import pytest

from streamfmt import decoded_codes, parse

hypothesis = pytest.importorskip("hypothesis")
from hypothesis import HealthCheck, given, settings  # noqa: E402
from hypothesis import strategies as st  # noqa: E402


def _leaf_sizes(n, r):
    """Leaf sizes left to right: a node of at most r particles is a leaf, else floor(c/2) go left."""
    return [n] if n <= r else _leaf_sizes(n >> 1, r) + _leaf_sizes(n - (n >> 1), r)


@st.composite
def inputs(draw):
    n = draw(st.integers(1, 400))
    kind = draw(st.sampled_from(["uniform", "grid", "clumps", "line"]))
    seed = draw(st.integers(0, 2**31 - 1))
    rng = np.random.default_rng(seed)
    scale = draw(st.sampled_from([1e-3, 1.0, 300.0, 1e5]))
    if kind == "uniform":
        pos = rng.uniform(-scale, scale, (n, 3))
    elif kind == "grid":  # many equal codes on every axis
        pos = rng.integers(0, 4, (n, 3)) * scale / 4
    elif kind == "clumps":
        c = rng.uniform(0, scale, (3, 3))
        pos = c[rng.integers(0, 3, n)] + rng.normal(0, scale / 100, (n, 3))
    else:  # collinear
        t = rng.uniform(0, scale, n)
        pos = np.stack([t, 2 * t, np.full(n, scale / 3)], 1)
    if n > 2 and draw(st.booleans()):  # exact duplicates
        pos[: n // 3] = pos[n // 3: 2 * (n // 3)]
    dtype = draw(st.sampled_from([np.float32, np.float64]))
    mode = draw(st.sampled_from(["abs", "rel"]))
    eb = draw(st.sampled_from([1e-1, 1e-2, 1e-3])) * (scale if mode == "abs" else 1.0)
    r = draw(st.sampled_from([1, 2, 3, 7, 16, 64, 500]))
    return pos.astype(dtype), mode, eb, r


@settings(max_examples=400, deadline=None, suppress_health_check=[HealthCheck.too_slow])
@given(inputs())
def test_oracle_properties(oracle_mod, case):
    pos, mode, eb, r = case
    n = pos.shape[0]
    m = oracle_mod.ABS if mode == "abs" else oracle_mod.REL
    b = oracle_mod.error_bound(pos, m, eb)
    stream, perm = oracle_mod.compress(pos, m, eb, leaf_size=r)
    s = parse(stream)
    assert s.n == n and np.array_equal(np.sort(perm), np.arange(n))
    assert [lf.count for lf in s.leaves] == _leaf_sizes(n, r)
    bits = 0
    for lf in s.leaves:
        w = sum(lf.m)
        bits += w * (lf.count - 1)
        for c in lf.codes:
            assert all(0 <= c[d] <= (1 << lf.m[d]) - 2 for d in range(3) if lf.m[d])
    assert s.payload_words == sum((sum(lf.m) * (lf.count - 1) + 31) // 32 for lf in s.leaves)
    assert bits <= 32 * s.payload_words < bits + 32 * len(s.leaves)
    q = oracle_mod.quantize(pos, m, eb)
    assert np.array_equal(decoded_codes(s), q[perm])
    dec = oracle_mod.decompress(stream)
    assert np.abs(pos[perm].astype(np.float64) - dec.astype(np.float64)).max() <= b.eps
    for red in (oracle_mod.compress_reduced(pos, m, eb, leaf_size=r)[:2], oracle_mod.reorder(stream, perm)[:2]):
        rs, rp = red
        assert np.array_equal(np.sort(rp), np.arange(n))
        assert np.abs(pos[rp].astype(np.float64) - oracle_mod.decompress(rs).astype(np.float64)).max() <= b.eps
