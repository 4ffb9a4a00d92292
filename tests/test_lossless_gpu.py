"""GPU parity of the lossless axes (Sec. 4.1: a dimension whose m_d would exceed
M is stored as the original coordinates).

Bounds far below what 30-bit codes can carry: float32 at a value-range-relative
bound of 1e-9 (eps under the float spacing of the data, so every axis is stored
losslessly) and float64 at 1e-12 (code ranges near 2^39 on every axis), slabs
where only the wide axis goes lossless, ragged sizes and leaf sizes.  Stream,
permutation and decoded floats must equal the oracle's byte for byte, and a
lossless axis must decode to the input bits.  The reduction, the reordering
and the leaf-size search refuse such inputs with the cause.
"""
import math

import numpy as np
import pytest

import synth
from test_parity_gpu import check_against_oracle, pc, run_gpu  # noqa: F401  (pc is a fixture)

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _check_lossless(pc, oracle_mod, pos, mode, eb, r, with_perm=True, expect_mask=None):
    got, info = check_against_oracle(pc, oracle_mod, pos, mode, eb, r, with_perm=with_perm)
    if expect_mask is not None:
        assert info.lossless_axes == expect_mask
    if pos.shape[0] and with_perm:
        _, perm, dec = run_gpu(pc, pos, mode, eb, r, True)
        for d in range(3):
            if info.lossless_axes >> d & 1:
                assert dec[:, d].tobytes() == pos[perm][:, d].tobytes()
    return info


@pytest.mark.parametrize("n,r", [(1 << 20, 4096), (300_001, 777), (65_537, 64), (150_000, 12000)])
def test_float32_bound_below_resolution(pc, oracle_mod, n, r):
    pos = synth.cosmology(n, seed=n, dtype=np.float32)
    _check_lossless(pc, oracle_mod, pos, pc.PC_EB_REL, 1e-9, r, expect_mask=7)


@pytest.mark.parametrize("n,r", [(1 << 19, 4096), (100_003, 1000)])
def test_float64_codes_beyond_thirty_bits(pc, oracle_mod, n, r):
    pos = synth.cosmology(n, seed=n, dtype=np.float64)
    _check_lossless(pc, oracle_mod, pos, pc.PC_EB_REL, 1e-12, r, expect_mask=7)


def test_float64_slab_wide_axis_only(pc, oracle_mod):
    rng = np.random.default_rng(1)
    n = 200_000
    pos = np.stack([rng.uniform(0, 1.0, n), rng.uniform(0, 1e-6, n), rng.uniform(0, 2e-6, n)], 1)
    _check_lossless(pc, oracle_mod, pos, pc.PC_EB_ABS, 1e-10, 2048, expect_mask=1)


def test_float32_slab_near_the_rounding_margin(pc, oracle_mod):
    """eps just above the rounding margin: the step is so small that x (range 1)
    needs codes of 2^30 or more while y and z (range 1e-5) stay coded."""
    rng = np.random.default_rng(7)
    n = 120_000
    pos = np.stack([rng.uniform(0, 1.0, n), rng.uniform(0, 1e-5, n), rng.uniform(-1e-5, 0, n)], 1).astype(np.float32)
    m = float(np.abs(pos.astype(np.float64)).max())

    def spacing(x, prec, emin):
        e = math.frexp(x)[1] - 1
        return math.ldexp(1.0, max(e, emin) - (prec - 1))

    eps = (spacing(2 * m, 24, -126) + 4 * spacing(2 * m, 53, -1022)) * 1.001
    assert oracle_mod.error_bound(pos, oracle_mod.ABS, eps).raw == 1
    _check_lossless(pc, oracle_mod, pos, pc.PC_EB_ABS, eps, 4096, expect_mask=1)


@pytest.mark.parametrize("n", [1, 2, 3, 4097, 8193, 40_000])
def test_ragged_sizes_without_and_with_perm(pc, oracle_mod, n):
    pos = synth.uniform(n, seed=n)
    mask = 7 if n > 1 else 0  # one particle: Delta_max = 0, every code 0 and exact (Sec. 3)
    _check_lossless(pc, oracle_mod, pos, pc.PC_EB_REL, 1e-9, 4096, with_perm=False, expect_mask=mask)
    _check_lossless(pc, oracle_mod, pos, pc.PC_EB_REL, 1e-9, 4096, with_perm=True, expect_mask=mask)


def test_next_rows_refuse_lossless_axes(pc):
    dev = torch.device("cuda:0")
    pos = torch.from_numpy(synth.cosmology(50_000, seed=4)).to(dev)
    for cfg in (pc.config(4096, reduce=True), pc.config(4096, reorder=True), pc.LEAF_AUTO):
        c = pc.Compressor(50_000, pc.PC_F32, leaf_size=cfg, device=dev)
        with pytest.raises(pc.PCError) as e:
            c.compress(pos, pc.PC_EB_REL, 1e-9)
        assert e.value.status == pc.PC_ERR_EB_TOO_SMALL
    pos64 = torch.from_numpy(synth.cosmology(50_000, seed=4, dtype=np.float64)).to(dev)
    c = pc.Compressor(50_000, pc.PC_F64, leaf_size=pc.config(4096, reduce=True), device=dev)
    with pytest.raises(pc.PCError) as e:
        c.compress(pos64, pc.PC_EB_REL, 1e-12)
    assert e.value.status == pc.PC_ERR_RANGE


def test_host_entry_points_and_batch(pc, oracle_mod):
    """The host-buffer entry points and the batch call take the same path."""
    n = 30_000
    pos = synth.cosmology(n, seed=9)
    ref, _ = oracle_mod.compress(pos, oracle_mod.REL, 1e-9)
    hp = torch.from_numpy(pos).pin_memory()
    ws = torch.empty(pc.pc_compress_host_workspace_size(n, pc.PC_F32), dtype=torch.uint8, device="cuda")
    hout = torch.empty(pc.pc_compress_bound(n, pc.PC_F32), dtype=torch.uint8).pin_memory()
    size = pc.pc_compress_host(hp, pc.PC_EB_REL, 1e-9, hout, ws)
    assert hout[:size].numpy().tobytes() == ref
    dev = torch.device("cuda:0")
    dpos = torch.from_numpy(pos).to(dev)
    out = torch.empty(pc.pc_compress_bound(n, pc.PC_F32), dtype=torch.uint8, device=dev)
    sizes, st = pc.pc_compress_batch([(dpos, pc.PC_EB_REL, 1e-9, 4096)], [out])
    assert list(st) == [pc.PC_OK] and out[: sizes[0]].cpu().numpy().tobytes() == ref
