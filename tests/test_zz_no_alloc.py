"""pc_compress_noalloc: compression for callers that may not allocate device memory.

Such callers (code inside another framework's memory pool, latency-critical
paths where cudaMalloc could synchronise the device) get the scratch from a
static 48 MiB device array in the library instead of a workspace argument.
The stream must be identical, byte for byte, to the one pc_compress writes,
on two calls in a row (the array keeps the previous call's contents).
"""
import ctypes

import numpy as np
import pytest

import synth

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


def reference_stream(pc, dpos, dtype, mode, eb, r):
    c = pc.Compressor(dpos.shape[0], dtype, leaf_size=r, device=dpos.device)
    size = c.compress(dpos, mode, eb)
    return c.out[:size].cpu().numpy().tobytes()


@pytest.mark.parametrize("gen,n,dtype,mode,eb,r", [
    ("uniform", 1 << 20, np.float32, "rel", 1e-3, 4096),
    ("cosmology", 300_001, np.float32, "rel", 1e-4, 777),
    ("fluid", 200_000, np.float64, "abs", 1e-4, 4096),
])
def test_noalloc_matches_pc_compress_twice(pc, gen, n, dtype, mode, eb, r):
    pos = synth.by_name(gen, n, seed=3, dtype=dtype)
    dev = torch.device("cuda:0")
    dpos = torch.from_numpy(pos).to(dev)
    pdt = pc.PC_F32 if dtype == np.float32 else pc.PC_F64
    m = pc.PC_EB_REL if mode == "rel" else pc.PC_EB_ABS
    ref = reference_stream(pc, dpos, pdt, m, eb, r)
    out = torch.empty(pc.pc_compress_bound(n, pdt, r), dtype=torch.uint8, device=dev)
    for _ in range(2):
        out.fill_(0xAB)
        size = pc.pc_compress_noalloc(dpos, m, eb, out, leaf_size=r)
        assert out[:size].cpu().numpy().tobytes() == ref


def test_noalloc_after_a_different_problem(pc):
    """A call after a larger, different call must not see its leftovers."""
    dev = torch.device("cuda:0")
    big = torch.from_numpy(synth.cosmology(900_000, seed=1)).to(dev)
    small = torch.from_numpy(synth.uniform(50_000, seed=2)).to(dev)
    out = torch.empty(pc.pc_compress_bound(900_000, pc.PC_F32), dtype=torch.uint8, device=dev)
    pc.pc_compress_noalloc(big, pc.PC_EB_REL, 1e-4, out)
    size = pc.pc_compress_noalloc(small, pc.PC_EB_REL, 1e-3, out)
    assert out[:size].cpu().numpy().tobytes() == reference_stream(pc, small, pc.PC_F32, pc.PC_EB_REL, 1e-3, 0)


def test_noalloc_rejects_problems_beyond_the_static_scratch(pc):
    n = 1 << 21
    assert pc.pc_compress_workspace_size(n, pc.PC_F32) > pc.PC_NOALLOC_SCRATCH_BYTES
    dev = torch.device("cuda:0")
    pos = torch.zeros((n, 3), dtype=torch.float32, device=dev)
    out = torch.empty(pc.pc_compress_bound(n, pc.PC_F32), dtype=torch.uint8, device=dev)
    with pytest.raises(pc.PCError) as e:
        pc.pc_compress_noalloc(pos, pc.PC_EB_REL, 1e-3, out)
    assert e.value.status == pc.PC_ERR_CAPACITY
    size = ctypes.c_uint64()
    rc = pc.load().pc_compress_noalloc(pos.data_ptr(), n, pc.PC_F32, pc.PC_EB_REL, 1e-3, None, out.data_ptr(),
                                       out.numel(), ctypes.byref(size), None)
    assert rc == pc.PC_ERR_CAPACITY


def test_noalloc_with_the_box_reduction(pc):
    """With PC_FLAG_BOX_REDUCTION the rounds go one launch at a time (no CUDA graph is
    instantiated for a caller that may not allocate); the stream is pc_compress's."""
    n = 300_000
    dev = torch.device("cuda:0")
    dpos = torch.from_numpy(synth.cosmology(n, seed=5)).to(dev)
    cfg = pc.config(2048, reduce=True)
    ref = reference_stream(pc, dpos, pc.PC_F32, pc.PC_EB_REL, 1e-3, cfg)
    out = torch.empty(pc.pc_compress_bound(n, pc.PC_F32, cfg), dtype=torch.uint8, device=dev)
    for _ in range(2):
        size = pc.pc_compress_noalloc(dpos, pc.PC_EB_REL, 1e-3, out, leaf_size=cfg)
        assert out[:size].cpu().numpy().tobytes() == ref
