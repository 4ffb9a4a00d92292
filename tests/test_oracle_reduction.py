"""Pins of the oracle's bit-box reduction (Sec. 4.1, Alg. 1, in rounds).

- An independent restatement of the round rule in plain Python on tiny inputs
  (boxes, selection, taken particles, rebuilt boxes, sequence order) gives the
  same sequences as the oracle; with one box per round (the least sum of m_d,
  lowest index on ties: Alg. 1's own order) it gives the oracle's
  one-per-round sequences, one round per sequence.
- Boxes that meet no other box: one round, and the stream is the plain one.
- Every particle is in exactly one sequence, every code fits its sequence's
  widths, and every decoded coordinate is within eps.
"""
import numpy as np
import pytest

import synth
from streamfmt import decoded_codes, parse


def _meet(a, b):
    return all(a["lo"][d] <= b["hi"][d] and b["lo"][d] <= a["hi"][d] for d in range(3))


def _box(oracle_mod, q, ids):
    c, lo, hi, qref, m = oracle_mod.bitbox(q[ids])
    h = [(1 << (int(md) - 1)) - 1 if md else 0 for md in m]
    return {"ids": list(ids), "centre": int(ids[c]), "qref": [int(x) for x in qref], "m": [int(x) for x in m],
            "key": int(sum(m)), "lo": [int(qref[d]) - h[d] for d in range(3)], "hi": [int(qref[d]) + h[d] for d in range(3)]}


def _reference_sequences(oracle_mod, pos, mode, eb, r, strict=False):
    """The reduction rule restated: returns [(centre id, qref, m, [ids in stream order])].
    strict: one box per round, the alive box of least (sum m_d, index), as Alg. 1 removes them."""
    q = oracle_mod.quantize(pos, mode, eb)
    order, loff, lcnt = oracle_mod.kdtree(q, r)
    boxes = [_box(oracle_mod, q, order[o: o + c]) for o, c in zip(loff, lcnt)]
    alive = [True] * len(boxes)
    seqs = []
    while any(alive):
        live = [i for i in range(len(boxes)) if alive[i]]
        if strict:
            sel = [min(live, key=lambda a: (boxes[a]["key"], a))]
        else:
            sel = [a for a in live if all(not (c != a and _meet(boxes[a], boxes[c])
                                               and (boxes[c]["key"], c) < (boxes[a]["key"], a)) for c in live)]
        lost = set()
        for a in sel:
            A = boxes[a]
            taken = []
            for c in live:
                if c == a or c in sel or not _meet(A, boxes[c]):
                    continue
                keep = []
                for pid in boxes[c]["ids"]:
                    if all(A["lo"][d] <= q[pid][d] <= A["hi"][d] for d in range(3)):
                        taken.append(pid)
                        lost.add(c)
                    else:
                        keep.append(pid)
                boxes[c]["ids"] = keep
            own = [pid for pid in A["ids"] if pid != A["centre"]]
            seqs.append((A["centre"], A["qref"], A["m"], [A["centre"]] + own + taken))
        for a in sel:
            alive[a] = False
        for c in lost:
            if boxes[c]["ids"]:
                boxes[c] = _box(oracle_mod, q, np.array(boxes[c]["ids"]))
            else:
                alive[c] = False
    return seqs


@pytest.mark.parametrize("gen,n,r,eb", [("cosmology", 400, 25, 1e-2), ("uniform", 300, 20, 5e-2),
                                        ("fluid", 500, 40, 1e-3), ("cosmology", 250, 7, 2e-2)])
def test_rounds_match_an_independent_restatement(oracle_mod, gen, n, r, eb):
    pos = synth.by_name(gen, n, seed=n + r)
    stream, perm, rounds = oracle_mod.compress_reduced(pos, oracle_mod.REL, eb, leaf_size=r)
    st = parse(stream)
    seqs = _reference_sequences(oracle_mod, pos, oracle_mod.REL, eb, r)
    assert st.num_leaves == len(seqs)
    for lf, (centre, qref, m, ids) in zip(st.leaves, seqs):
        assert tuple(lf.q_ref) == tuple(qref) and tuple(lf.m) == tuple(m)
        assert np.array_equal(perm[lf.particle_offset: lf.particle_offset + lf.count], ids)
    assert rounds >= 1


@pytest.mark.parametrize("gen,n,r,eb", [("cosmology", 300, 20, 1e-2), ("uniform", 200, 16, 5e-2),
                                        ("fluid", 360, 30, 1e-3)])
def test_one_box_per_round_matches_alg1_restated(oracle_mod, gen, n, r, eb):
    pos = synth.by_name(gen, n, seed=n + 2 * r)
    stream, perm, rounds = oracle_mod.compress_reduced(pos, oracle_mod.REL, eb, leaf_size=r, one_per_round=True)
    st = parse(stream)
    seqs = _reference_sequences(oracle_mod, pos, oracle_mod.REL, eb, r, strict=True)
    assert st.num_leaves == len(seqs) == rounds
    for lf, (centre, qref, m, ids) in zip(st.leaves, seqs):
        assert tuple(lf.q_ref) == tuple(qref) and tuple(lf.m) == tuple(m)
        assert np.array_equal(perm[lf.particle_offset: lf.particle_offset + lf.count], ids)
    assert np.array_equal(np.sort(perm), np.arange(n))
    b = oracle_mod.error_bound(pos, oracle_mod.REL, eb)
    assert np.abs(pos[perm].astype(np.float64) - oracle_mod.decompress(stream).astype(np.float64)).max() <= b.eps


def test_separated_boxes_give_the_plain_stream(oracle_mod):
    """Eight tight clusters at the corners of a cube, one per leaf: no box meets
    another, so one round emits the leaves in order."""
    rng = np.random.default_rng(5)
    corners = np.array([[x, y, z] for x in (0, 1000) for y in (0, 1000) for z in (0, 1000)], np.float64)
    pos = np.concatenate([c + rng.uniform(-1, 1, (512, 3)) for c in corners]).astype(np.float32)
    pos = pos[rng.permutation(len(pos))]
    plain, pperm = oracle_mod.compress(pos, oracle_mod.ABS, 0.01, leaf_size=512)
    red, rperm, rounds = oracle_mod.compress_reduced(pos, oracle_mod.ABS, 0.01, leaf_size=512)
    assert rounds == 1 and red == plain and np.array_equal(pperm, rperm)


@pytest.mark.parametrize("gen,n,r,mode,eb", [("cosmology", 60_000, 500, "rel", 1e-3),
                                             ("fluid", 40_000, 1000, "abs", 1e-3),
                                             ("uniform", 30_000, 300, "rel", 1e-2)])
def test_reduced_stream_is_valid(oracle_mod, gen, n, r, mode, eb):
    pos = synth.by_name(gen, n, seed=2)
    m = oracle_mod.ABS if mode == "abs" else oracle_mod.REL
    stream, perm, rounds = oracle_mod.compress_reduced(pos, m, eb, leaf_size=r)
    assert np.array_equal(np.sort(perm), np.arange(n))
    st = parse(stream)
    for lf in st.leaves:
        for c in lf.codes:
            assert all(c[d] <= (1 << lf.m[d]) - 2 for d in range(3) if lf.m[d])
    b = oracle_mod.error_bound(pos, m, eb)
    dec = oracle_mod.decompress(stream)
    assert np.abs(pos[perm].astype(np.float64) - dec.astype(np.float64)).max() <= b.eps
    assert np.array_equal(decoded_codes(st), oracle_mod.quantize(pos, m, eb)[perm])
    plain, _ = oracle_mod.compress(pos, m, eb, leaf_size=r)
    assert st.num_leaves <= parse(plain, with_codes=False).num_leaves


@pytest.mark.parametrize("gen,n,r,mode,eb", [("cosmology", 1 << 18, 2048, "rel", 1e-3),
                                             ("cosmology", 1 << 18, 2048, "rel", 1e-4),
                                             ("uniform", 1 << 17, 1024, "rel", 1e-3),
                                             ("fluid", 1 << 17, 1024, "abs", 1e-4)])
def test_rounds_stay_close_to_the_one_box_order(oracle_mod, gen, n, r, mode, eb):
    """The rounds reading of Alg. 1 (every box whose key is below that of every
    box it meets goes in the same round) against Alg. 1's own order (one box,
    least sum m_d, per round): both shrink the plain stream, and their sizes
    differ by at most 0.6 % (measured on these sets: 0.30 %, 0.06 %, 0.55 %,
    0.12 %; at 2^20 with r = 4096: 0.08 %, 0.35 %, 0.02 %)."""
    pos = synth.by_name(gen, n, seed=3)
    m = oracle_mod.ABS if mode == "abs" else oracle_mod.REL
    plain, _ = oracle_mod.compress(pos, m, eb, leaf_size=r, want_perm=False)
    rounds, _, nr = oracle_mod.compress_reduced(pos, m, eb, leaf_size=r, want_perm=False)
    one, _, n1 = oracle_mod.compress_reduced(pos, m, eb, leaf_size=r, want_perm=False, one_per_round=True)
    assert len(rounds) < len(plain) and len(one) < len(plain)
    assert nr < n1  # rounds take several boxes at once
    assert abs(len(rounds) / len(one) - 1.0) <= 0.006


def test_paper_box_length_holds_the_integer_range(oracle_mod):
    """Eq. 3 (bit box length): a bit box of m_d bits is l_d = 4 eps (2^(m_d - 1) - 0.5)
    long, centred at its centre particle, i.e. 2^(m_d - 1) - 0.5 lattice steps
    (2 eps) each side.  In doubled lattice units, to stay exact: the codes inside
    it are exactly those within 2^(m_d - 1) - 1 of the centre code (the integer
    range this library uses, reading 13); every particle of the leaf the oracle's
    bit box comes from is inside; two boxes share a lattice code exactly when
    their integer ranges overlap, and closed boxes one step further apart touch
    only between lattice codes."""
    rng = np.random.default_rng(13)

    def inside(x, c, m):  # Eq. 3, closed box, doubled units
        return 2 * abs(x - c) <= (1 << m) - 1 if m else x == c

    for _ in range(300):
        n = int(rng.integers(1, 40))
        q = rng.integers(0, 1 << int(rng.integers(1, 12)), (n, 3)).astype(np.int64)
        _, _, _, qref, m = oracle_mod.bitbox(q)
        for d in range(3):
            c, md = int(qref[d]), int(m[d])
            h = (1 << (md - 1)) - 1 if md else 0
            for x in range(c - h - 3, c + h + 4):
                assert inside(x, c, md) == (abs(x - c) <= h)
            assert all(inside(int(x), c, md) for x in q[:, d])
    for _ in range(2000):
        ma, mb = (int(v) for v in rng.integers(0, 8, 2))
        ha = (1 << (ma - 1)) - 1 if ma else 0
        hb = (1 << (mb - 1)) - 1 if mb else 0
        delta = int(rng.integers(0, ha + hb + 4))
        shared = any(inside(x, 0, ma) and inside(x, delta, mb) for x in range(-ha - 2, delta + hb + 3))
        assert shared == (delta <= ha + hb)
        # the closed real boxes: half-lengths ha + 1/2 and hb + 1/2 steps (a box of m_d = 0 is a point)
        touch = 2 * delta <= ((1 << ma) - 1 if ma else 0) + ((1 << mb) - 1 if mb else 0)
        if ma and mb:
            assert touch == (delta <= ha + hb + 1)
