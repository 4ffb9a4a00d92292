"""Failure detection on the GPU without a fault: the library's bounded wait
(the partition's wait on its tile copies) is run on a barrier that nothing
completes.  It must give up, report PC_ERR_TIMEOUT through the device error
word, and leave the context usable for the next call."""
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
    return pc


def test_bounded_wait_gives_up_and_the_context_survives(pc, oracle_mod):
    for _ in range(3):
        assert pc.pc_selftest_wait_timeout() == pc.PC_ERR_TIMEOUT
    pos = synth.cosmology(20_000, seed=3)
    c = pc.Compressor(pos.shape[0], pc.PC_F32, leaf_size=512, device=torch.device("cuda:0"))
    size = c.compress(torch.from_numpy(pos).cuda(), pc.PC_EB_REL, 1e-3)
    ref, _ = oracle_mod.compress(pos, oracle_mod.REL, 1e-3, leaf_size=512)
    assert c.out[:size].cpu().numpy().tobytes() == ref


@pytest.mark.parametrize("n", [1 << 20, 1 << 24])
def test_scatter_timeout_leaves_promptly(pc, oracle_mod, n):
    """A compress whose scatter tile copies never land (the self-test drops
    them; no copy is stuck): every scatter block gives up on its first tile
    after a short bounded wait and leaves, the later kernels see the error
    word and do nothing, and the call returns PC_ERR_TIMEOUT within well under
    a second.  The next plain call on the same workspace is byte-exact."""
    import time

    dev = torch.device("cuda:0")
    pos = torch.from_numpy(synth.cosmology(n, seed=5)).to(dev)
    ws = torch.empty(pc.pc_compress_workspace_size(n, pc.PC_F32), dtype=torch.uint8, device=dev)
    out = torch.empty(pc.pc_compress_bound(n, pc.PC_F32), dtype=torch.uint8, device=dev)
    times = []
    for _ in range(3):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        assert pc.pc_selftest_scatter_timeout(pos, out, ws) == pc.PC_ERR_TIMEOUT
        times.append(time.perf_counter() - t0)
    print(f"n={n}: scatter-timeout calls took {[round(t * 1e3, 2) for t in times]} ms")
    assert min(times) < 0.5
    small = pos[: 1 << 18]
    size = pc.pc_compress(small, pc.PC_EB_REL, 1e-3, out, ws)
    ref, _ = oracle_mod.compress(small.cpu().numpy(), oracle_mod.REL, 1e-3)
    assert out[:size].cpu().numpy().tobytes() == ref
