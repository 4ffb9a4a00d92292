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
