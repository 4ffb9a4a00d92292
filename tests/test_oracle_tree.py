"""Pins of the oracle's k-d partition (Sec. 4.1) against a second, independently
written recursive implementation (numpy lexsort per node) and against the
properties the paper states: median split, the median on the larger side,
leaves of at most r particles."""
import numpy as np
import pytest

import synth


def brute_tree(q, r):
    """Recursive full sort per node: returns the leaves as lists of original indices."""
    leaves = []

    def rec(ids, depth):
        if len(ids) <= r:
            leaves.append(sorted(ids))
            return
        axis = depth % 3
        ids = np.asarray(ids)
        order = np.lexsort((ids, q[ids, axis]))  # primary key: code, then original index
        k = len(ids) // 2
        rec(sorted(ids[order[:k]].tolist()), depth + 1)
        rec(sorted(ids[order[k:]].tolist()), depth + 1)

    if len(q):
        rec(list(range(len(q))), 0)
    return leaves


def tie_heavy(n, seed, levels=4):
    rng = np.random.default_rng(seed)
    return rng.integers(0, levels, (n, 3)).astype(np.int64)


INPUTS = [
    ("uniform", 1000, 7), ("uniform", 4096, 64), ("uniform", 3001, 1), ("uniform", 777, 2),
    ("ties", 2000, 33), ("ties", 4096, 5), ("ties", 129, 64), ("cosmology", 4000, 100), ("fluid", 3000, 50),
]


@pytest.mark.parametrize("kind,n,r", INPUTS)
def test_tree_matches_brute_force(oracle_mod, kind, n, r):
    if kind == "ties":
        q = tie_heavy(n, 3)
    else:
        pos = synth.by_name(kind, n, seed=1)
        q = oracle_mod.quantize(pos, oracle_mod.REL, 1e-3)
    order, off, cnt = oracle_mod.kdtree(q, r)
    want = brute_tree(q, r)
    got = [order[o:o + c].tolist() for o, c in zip(off, cnt)]
    assert got == want


@pytest.mark.parametrize("n,r", [(1, 1), (5, 5), (5, 4), (2 * 300 + 1, 300), (1 << 12, 1 << 9), (1000, 1000),
                                 (999, 1000), (4097, 4096), (3 * 4096 + 5, 4096)])
def test_tree_properties(oracle_mod, n, r):
    q = oracle_mod.quantize(synth.uniform(n, seed=n), oracle_mod.REL, 1e-3)
    order, off, cnt = oracle_mod.kdtree(q, r)
    assert np.array_equal(np.sort(order), np.arange(n))
    assert cnt.sum() == n and (cnt <= r).all() and (cnt >= 1).all()
    assert off[0] == 0 and np.array_equal(off[1:], np.cumsum(cnt)[:-1])
    # every leaf keeps increasing original index order
    for o, c in zip(off, cnt):
        seg = order[o:o + c]
        assert (np.diff(seg) > 0).all()
    if n <= r:
        assert len(cnt) == 1
    # node sizes at depth k are floor(n / 2^k) or ceil(n / 2^k)
    for c in cnt:
        ok = False
        for k in range(0, 40):
            lo, hi = n >> k, -(-n // (1 << k))
            if c in (lo, hi):
                ok = True
                break
        assert ok
    assert len(cnt) == oracle_mod.num_leaves(n, r)


def test_median_goes_right(oracle_mod):
    """Sec. 4.1: the median lies on the side with larger coordinates.  With an odd
    count the root's right child holds the median and one more particle."""
    q = np.array([[5, 0, 0], [1, 0, 0], [3, 0, 0], [4, 0, 0], [2, 0, 0]], np.int64)
    order, off, cnt = oracle_mod.kdtree(q, 3)
    assert cnt.tolist() == [2, 3]
    assert sorted(q[order[:2], 0].tolist()) == [1, 2]
    assert sorted(q[order[2:], 0].tolist()) == [3, 4, 5]


def test_ties_split_by_original_index(oracle_mod):
    """Equal codes on the split axis: the lower original indices go left."""
    q = np.zeros((8, 3), np.int64)
    order, off, cnt = oracle_mod.kdtree(q, 4)
    assert order[:4].tolist() == [0, 1, 2, 3] and order[4:].tolist() == [4, 5, 6, 7]


def test_left_keys_below_right_keys(oracle_mod):
    """At every split, every left particle precedes every right one in the
    (code, original index) order on that depth's axis."""
    q = tie_heavy(3000, 8, levels=6)
    r = 40
    order, off, cnt = oracle_mod.kdtree(q, r)

    def check(lo, hi, depth):
        n = hi - lo
        if n <= r:
            return
        k = n // 2
        ax = depth % 3
        left = order[lo:lo + k]
        right = order[lo + k:hi]
        lk = max(zip(q[left, ax], left))
        rk = min(zip(q[right, ax], right))
        assert lk < rk
        check(lo, lo + k, depth + 1)
        check(lo + k, hi, depth + 1)

    check(0, len(q), 0)


def brute_tree_widest(q, r):
    """The widest-cell rule written again: the root cell spans codes [0, max] per
    axis; a node splits on the axis of its widest cell (the lowest of equal
    widths) at the median code v, the left child's cell ending at v and the
    right child's starting there."""
    leaves = []

    def rec(ids, lo, hi):
        if len(ids) <= r:
            leaves.append(sorted(ids))
            return
        ext = [hi[d] - lo[d] for d in range(3)]
        axis = ext.index(max(ext))
        ids = np.asarray(ids)
        order = np.lexsort((ids, q[ids, axis]))
        k = len(ids) // 2
        v = int(q[ids[order[k]], axis])
        lhi, rlo = list(hi), list(lo)
        lhi[axis] = v
        rlo[axis] = v
        rec(sorted(ids[order[:k]].tolist()), lo, lhi)
        rec(sorted(ids[order[k:]].tolist()), rlo, hi)

    if len(q):
        rec(list(range(len(q))), [0, 0, 0], [int(q[:, d].max()) for d in range(3)])
    return leaves


@pytest.mark.parametrize("kind,n,r", INPUTS)
def test_widest_tree_matches_brute_force(oracle_mod, kind, n, r):
    if kind == "ties":
        q = tie_heavy(n, 3)
    else:
        pos = synth.by_name(kind, n, seed=1)
        q = oracle_mod.quantize(pos, oracle_mod.REL, 1e-3)
    order, off, cnt = oracle_mod.kdtree(q, r, widest=True)
    got = [order[o:o + c].tolist() for o, c in zip(off, cnt)]
    assert got == brute_tree_widest(q, r)


def test_widest_rule_follows_the_long_side(oracle_mod):
    """A slab 64 x 8 x 1 units: the first two cuts are both across x (halving x
    leaves 32 > 8), which depth mod 3 would not do, and the leaves differ."""
    rng = np.random.default_rng(4)
    pos = (rng.random((4096, 3)) * np.array([64.0, 8.0, 1.0])).astype(np.float32)
    q = oracle_mod.quantize(pos, oracle_mod.ABS, 0.01)
    order, off, cnt = oracle_mod.kdtree(q, 1024, widest=True)
    xs = [q[order[o:o + c], 0] for o, c in zip(off, cnt)]
    # four leaves, ordered along x: each leaf's x range lies below the next one's
    assert len(xs) == 4 and all(xs[i].max() <= xs[i + 1].min() for i in range(3))
    o2, f2, c2 = oracle_mod.kdtree(q, 1024)
    assert [order[o:o + c].tolist() for o, c in zip(off, cnt)] != [o2[o:o + c].tolist() for o, c in zip(f2, c2)]


def test_two_clusters_example_splits_the_larger_cluster(oracle_mod):
    """The paper's example of the median rule's limitation (golden file
    two_clusters_sec6.json): 100 particles in two clusters of 70 and 30 are split
    50 / 50, so 20 particles of the larger cluster go to the side of the smaller."""
    import json
    import os

    with open(os.path.join(os.path.dirname(__file__), "golden", "two_clusters_sec6.json")) as f:
        g = json.load(f)
    big, small = g["cluster_sizes"]
    rng = np.random.default_rng(70)
    a = np.column_stack([rng.normal(10.0, 1.0, big), rng.uniform(0, 1, big), rng.uniform(0, 1, big)])
    b = np.column_stack([rng.normal(200.0, 1.0, small), rng.uniform(0, 1, small), rng.uniform(0, 1, small)])
    pos = np.concatenate([a, b])
    shuffle = rng.permutation(g["n"])
    pos = pos[shuffle].astype(np.float32)
    in_big = shuffle < big  # particle i of the input came from the larger cluster
    q = oracle_mod.quantize(pos, oracle_mod.REL, 1e-4)
    order, off, cnt = oracle_mod.kdtree(q, g["n"] // 2)
    assert cnt.tolist() == g["first_split_sizes"]
    left, right = order[off[0]:off[0] + cnt[0]], order[off[1]:off[1] + cnt[1]]
    assert in_big[left].all()  # the smaller coordinates: only the larger cluster
    assert int(in_big[right].sum()) == big - g["first_split_sizes"][0] and int((~in_big[right]).sum()) == small
