"""The next rows of the method at a large size (cosmology 2^25, float32, rel eb
1e-4, r = 4096): the bit-box reduction, the reordering and the widest-cell split
axis, each alone and reduction + reordering together.  The oracle's reduction
is too slow at this size, so the checks are the properties that hold at any
size, computed on the GPU:
  * every decoded coordinate lies within eps of its input, through perm;
  * perm is a permutation of the input indices;
  * reordering keeps the stream size and the multiset of decoded particles of
    the unreordered stream;
  * the reduction writes at most as many sequences as there are leaves, and
    every sequence's codes fit its widths (the decoder validates the table).
"""
import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

N = 1 << 25
LEAF = 4096
EB = 1e-4


@pytest.fixture(scope="module")
def env():
    import paper_2404_02826_gb300 as pc
    from paper_2404_02826_gb300 import build as b

    b.build()
    pc.load()
    dev = torch.device("cuda:0")
    pos = torch.from_numpy(synth.cosmology(N, seed=0)).to(dev)
    return pc, dev, pos


def run(env, **flags):
    pc, dev, pos = env
    c = pc.Compressor(N, pc.PC_F32, leaf_size=pc.config(LEAF, **flags), with_perm=True, device=dev)
    size = c.compress(pos, pc.PC_EB_REL, EB)
    dec = torch.empty_like(pos)
    c.decompress(c.out, dec, size)
    torch.cuda.synchronize()
    info = pc.pc_stream_info(c.out[:96].cpu().numpy().tobytes())
    perm = c.perm[:N].long()
    return size, info, perm, dec


def check_bound_and_perm(env, info, perm, dec):
    _, _, pos = env
    assert torch.equal(torch.sort(perm).values, torch.arange(N, device=perm.device))
    err = (pos[perm].double() - dec.double()).abs().max().item()
    assert err <= info.eps


def sorted_rows(dec):
    # a canonical order of the decoded particles (their bits, lexicographically)
    b = dec.contiguous().view(torch.int32).long()
    key = (b[:, 0] << 32 | (b[:, 1] & 0xffffffff))
    order = torch.argsort(b[:, 2], stable=True)
    order = order[torch.argsort(key[order], stable=True)]
    return dec[order]


@pytest.mark.parametrize("flags", [dict(reduce=True), dict(widest=True), dict(reduce=True, reorder=True)])
def test_next_rows_decode_within_eps(env, flags):
    size, info, perm, dec = run(env, **flags)
    check_bound_and_perm(env, info, perm, dec)
    if flags.get("reduce"):
        assert info.num_leaves <= N // LEAF
    else:
        assert info.num_leaves == N // LEAF


def test_reordering_keeps_size_and_particles(env):
    size0, info0, _, dec0 = run(env)
    size1, info1, perm1, dec1 = run(env, reorder=True)
    check_bound_and_perm(env, info1, perm1, dec1)
    assert size1 == size0 and info1.num_leaves == info0.num_leaves
    assert torch.equal(sorted_rows(dec0), sorted_rows(dec1))
