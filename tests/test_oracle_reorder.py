"""Pins of the oracle's reordering for the entropy coder (Sec. 4.2, after Fig. 4).

- The paper's two examples: the R-index of (01, 100111, 01010) with the axes
  ordered x, z, y, and that axis order from the m_d distributions it describes.
- An independent restatement in plain Python (entropy with math.log2, Python
  sorts, bit-by-bit re-encoding) writes the same bytes.
- Invariants: every sequence keeps its particles (the same decoded set) and its
  record fields; sequences ascend in sum m_d and particles in R-index; the
  result is a fixed point; perm follows the particles.
"""
import json
import math
import os

import numpy as np
import pytest

import synth
from streamfmt import parse

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
AX = {"x": 0, "y": 1, "z": 2}


def test_rindex_example(oracle_mod):
    g = json.load(open(os.path.join(GOLDEN, "rindex_example_sec4_2.json")))
    c = [int(g["codes"][a], 2) for a in "xyz"]
    m = [len(g["codes"][a]) for a in "xyz"]
    order = [AX[a] for a in g["axis_order"]]
    r = oracle_mod.rindex(c, m, order)
    assert format(r, "0{}b".format(sum(m))) == g["rindex"]


def test_axis_order_example(oracle_mod):
    g = json.load(open(os.path.join(GOLDEN, "axis_entropy_example_sec4_2.json")))
    rows = []
    peak = {2: 1, 3: 3, 4: 10, 5: 40, 6: 10, 7: 3, 8: 1, 9: 1}  # one peak, support 2..9
    zs = [v for v, k in peak.items() for _ in range(k)]
    for i in range(len(zs) * 24):
        rows.append((2 + i % 3, 2 + (i // 3) % 8, zs[i % len(zs)]))
    order, ent = oracle_mod.axis_order(np.array(rows))
    assert order == tuple(AX[a] for a in g["axis_order"])
    assert abs(ent[0] - math.log2(3)) < 1e-12 and abs(ent[1] - 3.0) < 1e-12


def _entropy(vals):
    n = len(vals)
    h = 0.0
    for v in set(vals):
        p = vals.count(v) / n
        h -= p * math.log2(p)
    return h


def _restated(stream):
    """Sec. 4.2 reordering written again from the stream: a second, plain Python implementation."""
    st = parse(stream)
    ms = [lf.m for lf in st.leaves]
    ent = [_entropy([m[d] for m in ms]) for d in range(3)]
    order = [0, 1, 2]
    for i in (1, 2):  # stable insertion sort; entropies within 1e-9 tie
        j = i
        while j > 0 and ent[order[j]] < ent[order[j - 1]] - 1e-9:
            order[j], order[j - 1] = order[j - 1], order[j]
            j -= 1
    seqs = sorted(range(st.num_leaves), key=lambda k: (sum(st.leaves[k].m), k))
    header = bytearray(stream[:96])
    table = bytearray()
    bits = 0
    nbits = 0
    words = 0
    off = 0
    for k in seqs:
        lf = st.leaves[k]
        recs = list(enumerate(lf.codes, start=1))

        def rix(c):
            r = 0
            for a in order:
                r = (r << lf.m[a]) | c[a]
            return r
        recs.sort(key=lambda ic: (rix(ic[1]), ic[0]))
        rec = bytearray(stream[96 + 32 * k: 96 + 32 * k + 32])
        rec[0:8] = off.to_bytes(8, "little")
        rec[8:16] = words.to_bytes(8, "little")
        table += rec
        for _, c in recs:
            for d in range(3):
                bits |= c[d] << nbits
                nbits += lf.m[d]
        w = sum(lf.m) * (lf.count - 1)
        nbits = (words + (w + 31) // 32) * 32  # next sequence starts on a fresh word
        words += (w + 31) // 32
        off += lf.count
    payload = bits.to_bytes(4 * words, "little") if words else b""
    return bytes(header + table + payload), tuple(order)


@pytest.mark.parametrize("gen,n,r,eb", [("cosmology", 3000, 100, 1e-3), ("uniform", 2000, 64, 1e-2),
                                        ("fluid", 2500, 300, 1e-4), ("cosmology", 700, 1, 1e-2)])
def test_reorder_matches_restatement(oracle_mod, gen, n, r, eb):
    pos = synth.by_name(gen, n, seed=n)
    stream, _ = oracle_mod.compress(pos, oracle_mod.REL, eb, leaf_size=r)
    got, _, order = oracle_mod.reorder(stream)
    ref, ref_order = _restated(stream)
    assert order == ref_order
    assert got == ref


@pytest.mark.parametrize("reduced", [False, True])
def test_reorder_invariants(oracle_mod, reduced):
    pos = synth.cosmology(40_000, seed=9)
    if reduced:
        stream, perm, _ = oracle_mod.compress_reduced(pos, oracle_mod.REL, 1e-3, leaf_size=500)
    else:
        stream, perm = oracle_mod.compress(pos, oracle_mod.REL, 1e-3, leaf_size=500)
    got, gperm, order = oracle_mod.reorder(stream, perm)
    assert len(got) == len(stream) and got[:96] == stream[:96]
    a, b = parse(stream), parse(got)
    seqs = sorted(range(a.num_leaves), key=lambda k: (sum(a.leaves[k].m), k))
    assert [sum(lf.m) for lf in b.leaves] == sorted(sum(lf.m) for lf in a.leaves)
    for k, lf in zip(seqs, b.leaves):
        old = a.leaves[k]
        assert (lf.q_ref, lf.m, lf.count) == (old.q_ref, old.m, old.count)
        assert sorted(lf.codes) == sorted(old.codes)
        rix = [oracle_mod.rindex(c, lf.m, order) for c in lf.codes]
        assert rix == sorted(rix)
    dec = oracle_mod.decompress(got)
    eps = oracle_mod.error_bound(pos, oracle_mod.REL, 1e-3).eps
    assert np.abs(pos[gperm].astype(np.float64) - dec).max() <= eps
    again, _, _ = oracle_mod.reorder(got)
    assert again == got
