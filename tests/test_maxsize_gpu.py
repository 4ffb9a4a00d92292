"""The largest input the library takes: n = PC_MAX_PARTICLES = 2^31 - 1
particles (an odd count, so the nodes of every level have floor and ceil of
n / 2^k particles), float32, uniform in a 1000^3 box, absolute eb 0.05, leaf
size 4096: 2^19 leaves of 4095 or 4096 particles.  About 160 GB of device
memory (input, output stream bound, workspace with input indices, decoded
copy); every check runs in chunks on the device.

What is checked (by what holds at any size, and by samples the oracle
computes one at a time):
  * the header's eps, s and origin equal the oracle's error bound of the
    input (Sec. 3); the leaf table's offsets follow the median rule's sizes
    (the left child of c particles gets floor(c / 2), Sec. 4.1);
  * every decoded coordinate lies within eps of its input, and the output
    permutation holds every input index once;
  * the first three levels (axes x, y, z): in every node the left half
    precedes the right half in (code, original index) order;
  * 16 sampled leaves: the oracle's bit box (Eq. 2) of the leaf's particles
    equals the leaf record, and the packed codes equal q - q_ref + 2^(m-1) - 1.
"""
import os
import struct

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

LEAF = 4096
LEVELS = 19  # the least depth with ceil(n / 2^depth) <= 4096
EB = 0.05
BOX = 1000.0
CHUNK = 1 << 27


def uniform_f32(n, seed):
    """n x 3 float32 uniform in [0, BOX), written chunk by chunk (no float64 copy)."""
    rng = np.random.default_rng(seed)
    out = np.empty((n, 3), np.float32)
    flat = out.reshape(-1)
    for a in range(0, flat.size, 1 << 28):
        v = flat[a: a + (1 << 28)]
        rng.random(out=v, dtype=np.float32)
        v *= np.float32(BOX)
    return out


def node_sizes(n, depth):
    """Sizes of the 2^depth nodes at `depth`, left to right: a node of c particles has children floor(c/2), rest."""
    c = np.array([n], np.int64)
    for _ in range(depth):
        left = c >> 1
        c = np.stack([left, c - left], 1).reshape(-1)
    return c


@pytest.fixture(scope="module")
def run():
    import paper_2404_02826_gb300 as pc
    from paper_2404_02826_gb300 import build as b

    b.build()
    pc.load()
    n = pc.PC_MAX_PARTICLES
    dev = torch.device("cuda:0")
    # device: input and decoded copy, stream bound, workspaces, permutation; host: the input
    need = (2 * 12 * n + pc.pc_compress_bound(n, pc.PC_F32, LEAF) + pc.pc_decompress_workspace_size(n)
            + pc.pc_compress_workspace_size(n, pc.PC_F32, LEAF, True) + 4 * n + (16 << 30))
    torch.cuda.empty_cache()  # earlier modules' cached blocks
    free, _ = torch.cuda.mem_get_info(dev)
    if free < need:
        pytest.skip(f"needs {need >> 30} GiB of device memory, {free >> 30} GiB free")
    if os.sysconf("SC_PAGE_SIZE") * os.sysconf("SC_PHYS_PAGES") < 3 * 12 * n:
        pytest.skip("not enough host memory for the input")
    pos_h = uniform_f32(n, seed=3)
    pos = torch.from_numpy(pos_h).to(dev)
    c = pc.Compressor(n, pc.PC_F32, leaf_size=LEAF, with_perm=True, device=dev)
    size = c.compress(pos, pc.PC_EB_ABS, EB)
    dec = torch.empty_like(pos)
    c.decompress(c.out, dec, size)
    torch.cuda.synchronize()
    info = pc.pc_stream_info(c.out[:96].cpu().numpy().tobytes())
    yield pc, n, info, pos_h, pos, c.out[:size], c.perm[:n], dec
    del c, pos, dec
    torch.cuda.empty_cache()


def test_header_and_leaf_table(run, oracle_mod):
    pc, n, info, pos_h, _, stream, _, _ = run
    b = oracle_mod.error_bound(pos_h, oracle_mod.ABS, EB)
    assert info.n == n and info.eps == b.eps and info.s == b.s and tuple(info.o) == tuple(b.o)
    sizes = node_sizes(n, LEVELS)
    assert info.num_leaves == sizes.size == 1 << LEVELS and set(np.unique(sizes).tolist()) == {LEAF - 1, LEAF}
    recs = np.frombuffer(stream[96: 96 + 32 * info.num_leaves].cpu().numpy().tobytes(), np.uint64).reshape(-1, 4)
    assert np.array_equal(recs[:, 0].astype(np.int64), np.concatenate([[0], np.cumsum(sizes)[:-1]]))


def test_every_coordinate_within_eps(run):
    _, n, info, _, pos, _, perm, dec = run
    seen = torch.zeros(n, dtype=torch.bool, device=pos.device)
    worst = 0.0
    for a in range(0, n, CHUNK):
        p = perm[a: a + CHUNK].long()
        seen[p] = True
        worst = max(worst, (pos[p].double() - dec[a: a + CHUNK].double()).abs().max().item())
    assert worst <= info.eps
    assert bool(seen.all())


def test_first_three_levels(run):
    _, n, info, _, pos, _, perm, _ = run

    def keys(a, b, axis):  # (code << 32 | original index) of output positions [a, b)
        p = perm[a:b].long()
        q = torch.round((pos[p, axis].double() - info.o[axis]) / info.s).long()  # half to even, as rint
        return (q << 32) | p

    def extreme(a, b, axis, hi):
        out = None
        for x in range(a, b, CHUNK):
            k = keys(x, min(b, x + CHUNK), axis)
            v = (k.max() if hi else k.min()).item()
            out = v if out is None else (max(out, v) if hi else min(out, v))
        return out

    for level in range(3):
        bounds = np.concatenate([[0], np.cumsum(node_sizes(n, level + 1))])
        for j in range(1 << level):
            lo, mid, hi = (int(x) for x in bounds[2 * j: 2 * j + 3])
            assert extreme(lo, mid, level, True) < extreme(mid, hi, level, False), f"level {level} node {j}"


def test_sampled_leaves_against_oracle(run, oracle_mod):
    _, n, info, pos_h, _, stream, perm, _ = run
    L = info.num_leaves
    head = stream[: 96 + 32 * L].cpu().numpy().tobytes()
    sizes = node_sizes(n, LEVELS)
    words = stream[96 + 32 * L:].cpu().numpy().view("<u4")
    rng = np.random.default_rng(4)
    for leaf in sorted(rng.choice(L, 16, replace=False)):
        po, wo, qx, qy, qz, mx, my, mz, z = struct.unpack_from("<QQiii4B", head, 96 + 32 * int(leaf))
        cnt = int(sizes[leaf])
        idx = perm[po: po + cnt].cpu().numpy().astype(np.int64)  # centre first, then the rest in leaf order
        order = np.sort(idx)  # leaf order: every partition is stable
        q = oracle_mod.quantize_on(pos_h[order], info.o, info.s)
        cpos, lo, hi, qref, m = oracle_mod.bitbox(q)
        assert np.array_equal(idx, np.concatenate([order[cpos:cpos + 1], np.delete(order, cpos)]))
        assert tuple(qref) == (qx, qy, qz) and tuple(m) == (mx, my, mz) and z == 0
        others = np.delete(q, cpos, axis=0)
        w = mx + my + mz
        nwords = (w * (cnt - 1) + 31) // 32
        bits = np.unpackbits(words[wo: wo + nwords].view(np.uint8), bitorder="little").astype(np.int64)
        start = 0
        for d, md in enumerate((mx, my, mz)):
            if md:
                at = np.arange(cnt - 1)[:, None] * w + start + np.arange(md)[None, :]
                got = (bits[at] << np.arange(md)[None, :]).sum(1)
                want = others[:, d] - (qx, qy, qz)[d] + (1 << (md - 1)) - 1
                assert np.array_equal(got, want)
            start += md
