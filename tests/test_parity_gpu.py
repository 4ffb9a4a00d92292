"""GPU parity: the CUDA path, called through the C ABI, against the oracle.

Integer and byte results must be identical: the whole stream (header, leaf
table = partition + bit boxes, packed codes), the permutation, and the decoded
floats (the oracle decodes with the same double-precision rule).  Every
decoded coordinate must lie within eps of its input.
"""
import struct

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


def run_gpu(pc, pos, mode, eb, r, with_perm=True):
    dev = torch.device("cuda:0")
    dpos = torch.from_numpy(np.ascontiguousarray(pos)).to(dev)
    dtype = pc.PC_F32 if pos.dtype == np.float32 else pc.PC_F64
    c = pc.Compressor(pos.shape[0], dtype, leaf_size=r, with_perm=with_perm, device=dev)
    size = c.compress(dpos, mode, eb)
    stream = c.out[:size].clone()
    out = torch.empty_like(dpos)
    if pos.shape[0]:
        c.decompress(stream, out, size)
    torch.cuda.synchronize()
    perm = c.perm[: pos.shape[0]].cpu().numpy().astype(np.int64) if with_perm else None
    return stream.cpu().numpy().tobytes(), perm, out.cpu().numpy()


def check_against_oracle(pc, oracle_mod, pos, mode, eb, r, with_perm=True):
    omode = oracle_mod.ABS if mode == pc.PC_EB_ABS else oracle_mod.REL
    ref_stream, ref_perm = oracle_mod.compress(pos, omode, eb, leaf_size=r)
    got_stream, perm, dec = run_gpu(pc, pos, mode, eb, r, with_perm)
    assert len(got_stream) == len(ref_stream)
    if got_stream != ref_stream:
        a = np.frombuffer(got_stream, np.uint8)
        b = np.frombuffer(ref_stream, np.uint8)
        first = int(np.flatnonzero(a != b)[0])
        raise AssertionError(f"stream differs from the oracle at byte {first} of {len(a)}")
    if with_perm:
        assert np.array_equal(perm, ref_perm)
    ref_dec = oracle_mod.decompress(ref_stream)
    assert dec.tobytes() == ref_dec.tobytes()
    info = pc.pc_stream_info(got_stream[:96])
    if pos.shape[0]:
        err = np.abs(pos[ref_perm].astype(np.float64) - dec.astype(np.float64))
        assert int((err > info.eps).sum()) == 0
    return got_stream, info


CONFIGS = [
    # generator, n, dtype, mode, eb, leaf size
    ("uniform", 1 << 20, np.float32, "rel", 1e-3, 4096),       # first workload, full size
    ("uniform", 100_000, np.float32, "rel", 1e-4, 4096),
    ("cosmology", 1 << 18, np.float32, "rel", 1e-4, 4096),
    ("cosmology", 1 << 18, np.float32, "rel", 1e-3, 4096),
    ("cosmology", 300_001, np.float32, "rel", 1e-3, 777),
    ("fluid", 1 << 18, np.float64, "abs", 1e-4, 4096),
    ("fluid", 100_003, np.float64, "abs", 1e-6, 1000),         # codes above 2^16 (u32 path)
    ("fluid", 70_000, np.float32, "abs", 1e-4, 4096),
    ("cosmology", 200_000, np.float64, "rel", 1e-7, 2048),      # u32 codes, float64
    ("uniform", 65_537, np.float32, "abs", 0.5, 64),            # many leaves, deep subtrees
    ("uniform", 40_000, np.float32, "rel", 1e-3, 1),            # one particle per leaf
    ("uniform", 33_000, np.float32, "rel", 1e-3, 2),
    ("cosmology", 150_000, np.float32, "rel", 1e-4, 12000),     # largest leaf size
]


@pytest.mark.parametrize("gen,n,dtype,mode,eb,r", CONFIGS)
def test_parity_generators(pc, oracle_mod, gen, n, dtype, mode, eb, r):
    pos = synth.by_name(gen, n, seed=5, dtype=dtype)
    m = pc.PC_EB_ABS if mode == "abs" else pc.PC_EB_REL
    check_against_oracle(pc, oracle_mod, pos, m, eb, r)


def test_parity_fluid_workload_full_size(pc, oracle_mod):
    """The fluid workload at its full size, as bench.py generates and runs it (2^24 float64
    lattice, seed 0, absolute eb 1e-4, leaf size 4096): the whole stream, the permutation
    and the decoded floats byte for byte."""
    pos = synth.by_name("fluid", 1 << 24, seed=0, dtype=np.float64)
    _, info = check_against_oracle(pc, oracle_mod, pos, pc.PC_EB_ABS, 1e-4, 4096)
    assert info.n == 1 << 24 and info.num_leaves == 1 << 12


@pytest.mark.parametrize("n", [0, 1, 2, 3, 5, 31, 32, 33, 1000, 4095, 4096, 4097, 8193, 16383, 16384, 16385,
                               32767, 32768, 32769, 65536 + 17, 131072 * 3 + 1])
def test_parity_ragged_sizes(pc, oracle_mod, n):
    pos = synth.uniform(n, seed=n)
    check_against_oracle(pc, oracle_mod, pos, pc.PC_EB_REL, 1e-3, 4096)


@pytest.mark.parametrize("n,r", [(5000, 4), (20000, 100), (70000, 333), (2 * 4096 + 1, 4096), (3 * 12000 + 7, 12000)])
def test_parity_leaf_sizes(pc, oracle_mod, n, r):
    pos = synth.cosmology(n, seed=r)
    check_against_oracle(pc, oracle_mod, pos, pc.PC_EB_REL, 1e-3, r)


@pytest.mark.parametrize("levels", [1, 3, 17])
def test_parity_heavy_ties(pc, oracle_mod, levels):
    """Integer-grid inputs: many equal codes on every split axis."""
    rng = np.random.default_rng(levels)
    pos = rng.integers(0, levels, (90_000, 3)).astype(np.float32)
    pos[0] = 0
    pos[1] = max(levels - 1, 1)
    check_against_oracle(pc, oracle_mod, pos, pc.PC_EB_ABS, 0.2, 500)


def test_parity_identical_and_collinear(pc, oracle_mod):
    same = np.tile(np.array([[1.5, -2.0, 7.25]], np.float32), (50_000, 1))
    check_against_oracle(pc, oracle_mod, same, pc.PC_EB_REL, 1e-3, 4096)
    x = np.random.default_rng(3).uniform(0, 9, 60_000)
    line = np.stack([x, np.full_like(x, 2.0), np.full_like(x, -1.0)], 1).astype(np.float32)
    check_against_oracle(pc, oracle_mod, line, pc.PC_EB_ABS, 1e-3, 1000)


@pytest.mark.parametrize("dtype", [np.float32, np.float64])
def test_parity_near_rounding_ties(pc, oracle_mod, dtype):
    """Coordinates on and next to lattice midpoints, so that round-half-even and
    the exact double-precision fallback of the quantizer decide the codes."""
    eps = 0.05
    corners = np.array([[0.0, 0.0, 0.0], [12.0, 12.0, 12.0]], dtype)
    b = oracle_mod.error_bound(corners, oracle_mod.ABS, eps)
    pts = synth.near_ties(80_000, b.o, b.s, seed=9, dtype=dtype, spread=int(12.0 / b.s) - 1)
    pos = np.concatenate([corners, pts]).astype(dtype)
    check_against_oracle(pc, oracle_mod, pos, pc.PC_EB_ABS, eps, 4096)


def test_parity_float32_exact_division_path(pc, oracle_mod):
    """float32 input whose codes exceed 2^22, so the quantizer divides in double."""
    pos = synth.uniform(50_000, seed=4, box=1.0)
    eps = 1.1 * 2.0 ** -22
    check_against_oracle(pc, oracle_mod, pos, pc.PC_EB_ABS, eps, 4096)


def test_parity_float64_wide_codes(pc, oracle_mod):
    """float64 input with codes near 2^29: the quantizer's rounding from the
    bits of (p - o) * (1/s) at its widest, and its division fallback."""
    pos = synth.uniform(50_000, seed=6, box=1.0, dtype=np.float64)
    check_against_oracle(pc, oracle_mod, pos, pc.PC_EB_ABS, 1e-9, 4096)


@pytest.mark.parametrize("gen,n,dtype,mode,eb", [
    ("cosmology", 300_000, np.float32, "rel", 1e-4),
    ("uniform", 200_003, np.float32, "rel", 1e-3),
    ("fluid", 150_000, np.float64, "abs", 1e-4),
])
def test_autotuned_leaf_size(pc, oracle_mod, gen, n, dtype, mode, eb):
    """The autotuned stream is the oracle's stream at the leaf size it records,
    and that leaf size is a local minimum of the stream size over the candidate
    depths (ceil(n / 2^d) between PC_AUTOTUNE_MIN_LEAF and PC_MAX_LEAF_SIZE)."""
    pos = synth.by_name(gen, n, seed=11, dtype=dtype)
    m = pc.PC_EB_ABS if mode == "abs" else pc.PC_EB_REL
    om = oracle_mod.ABS if mode == "abs" else oracle_mod.REL
    got, perm, dec = run_gpu(pc, pos, m, eb, pc.LEAF_AUTO)
    r = pc.pc_stream_info(got[:96]).leaf_size
    ref, ref_perm = oracle_mod.compress(pos, om, eb, leaf_size=r)
    assert got == ref and np.array_equal(perm, ref_perm)
    assert dec.tobytes() == oracle_mod.decompress(ref).tobytes()
    ceil_at = lambda d: -(-n // (1 << d))
    depths = [d for d in range(40) if ceil_at(d) <= pc.PC_MAX_LEAF_SIZE]
    first = depths[0]
    cands = [first] + [d for d in depths[1:] if ceil_at(d) >= pc.PC_AUTOTUNE_MIN_LEAF]
    chosen = [d for d in cands if ceil_at(d) == r]
    assert len(chosen) == 1
    d = chosen[0]
    size = len(ref)
    if d - 1 in cands:
        assert len(oracle_mod.compress(pos, om, eb, leaf_size=ceil_at(d - 1), want_perm=False)[0]) > size
    if d + 1 in cands:
        assert len(oracle_mod.compress(pos, om, eb, leaf_size=ceil_at(d + 1), want_perm=False)[0]) >= size


def test_leaf_size_sweep_matches_oracle_sizes(pc, oracle_mod):
    """Every sweep point is the size of the oracle's stream at that leaf size,
    split into header, leaf table and packed codes; the autotuned stream is the
    first point whose successor is not smaller."""
    pos = synth.cosmology(200_000, seed=21)
    dpos = torch.from_numpy(pos).cuda()
    pts = pc.pc_leaf_size_sweep(dpos, pc.PC_EB_REL, 1e-4, r_min=256, r_max=12000)
    assert [p["leaf_size"] for p in pts] == sorted((p["leaf_size"] for p in pts), reverse=True)
    assert pts[0]["leaf_size"] <= 12000 and pts[-1]["leaf_size"] >= 256
    for p in pts:
        ref, _ = oracle_mod.compress(pos, oracle_mod.REL, 1e-4, leaf_size=p["leaf_size"], want_perm=False)
        n, _, nl, nw = oracle_mod.stream_header(ref)
        assert p["total_bytes"] == len(ref)
        assert p["leaves"] == nl and p["table_bytes"] == 32 * nl and p["payload_bytes"] == 4 * nw
    auto = pc.pc_leaf_size_sweep(dpos, pc.PC_EB_REL, 1e-4, r_min=pc.PC_AUTOTUNE_MIN_LEAF, r_max=12000)
    got, _, _ = run_gpu(pc, pos, pc.PC_EB_REL, 1e-4, pc.LEAF_AUTO, with_perm=False)
    k = 0
    while k + 1 < len(auto) and auto[k + 1]["total_bytes"] < auto[k]["total_bytes"]:
        k += 1
    assert len(got) == auto[k]["total_bytes"]
    assert pc.pc_stream_info(got[:96]).leaf_size == auto[k]["leaf_size"]


def test_parity_without_perm(pc, oracle_mod):
    pos = synth.cosmology(120_000, seed=8)
    check_against_oracle(pc, oracle_mod, pos, pc.PC_EB_REL, 1e-4, 4096, with_perm=False)


def test_unaligned_input(pc, oracle_mod):
    pos = synth.uniform(20_001, seed=12)
    dev = torch.device("cuda:0")
    big = torch.from_numpy(pos).to(dev)
    view = big[1:]  # 12-byte offset: not 16-byte aligned
    c = pc.Compressor(view.shape[0], pc.PC_F32, device=dev)
    size = c.compress(view, pc.PC_EB_REL, 1e-3)
    ref, _ = oracle_mod.compress(pos[1:], oracle_mod.REL, 1e-3)
    assert c.out[:size].cpu().numpy().tobytes() == ref


def test_status_codes(pc):
    dev = torch.device("cuda:0")
    pos = torch.rand(1000, 3, device=dev)
    c = pc.Compressor(1000, pc.PC_F32, device=dev)
    bad = pos.clone()
    bad[17, 2] = float("nan")
    with pytest.raises(pc.PCError) as e:
        c.compress(bad, pc.PC_EB_REL, 1e-3)
    assert e.value.status == pc.PC_ERR_NONFINITE
    bad[17, 2] = float("inf")
    with pytest.raises(pc.PCError) as e:
        c.compress(bad, pc.PC_EB_REL, 1e-3)
    assert e.value.status == pc.PC_ERR_NONFINITE
    for eb in (0.0, -1.0, float("nan")):
        with pytest.raises(pc.PCError) as e:
            c.compress(pos, pc.PC_EB_REL, eb)
        assert e.value.status == pc.PC_ERR_ARG
    # eps below the float spacing of the data: stored losslessly (Sec. 4.1, m_d > M),
    # refused by the bit-box reduction, which needs codes
    far = torch.tensor([[1e6, 0, 0], [1e6 + 64, 1, 1]], device=dev)
    c2 = pc.Compressor(2, pc.PC_F32, device=dev)
    size2 = c2.compress(far, pc.PC_EB_ABS, 1e-3)
    assert pc.pc_stream_info(c2.out[:96].cpu().numpy().tobytes()).lossless_axes == 7
    back = torch.empty_like(far)
    c2.decompress(c2.out, back, size2)
    assert sorted(map(tuple, back.cpu().tolist())) == sorted(map(tuple, far.cpu().tolist()))
    c3 = pc.Compressor(2, pc.PC_F32, leaf_size=pc.config(4096, reduce=True), device=dev)
    with pytest.raises(pc.PCError) as e:
        c3.compress(far, pc.PC_EB_ABS, 1e-3)
    assert e.value.status == pc.PC_ERR_EB_TOO_SMALL
    small_out = torch.empty(100, dtype=torch.uint8, device=dev)
    with pytest.raises(pc.PCError) as e:
        pc.pc_compress(pos, pc.PC_EB_REL, 1e-3, small_out, c.ws)
    assert e.value.status == pc.PC_ERR_CAPACITY


def test_corrupt_streams_are_rejected(pc, oracle_mod):
    pos = synth.cosmology(50_000, seed=21)
    stream, _ = oracle_mod.compress(pos, oracle_mod.REL, 1e-3, leaf_size=1000)
    dev = torch.device("cuda:0")
    ws = torch.empty(pc.pc_decompress_workspace_size(50_000), dtype=torch.uint8, device=dev)
    out = torch.empty((50_000, 3), dtype=torch.float32, device=dev)

    def attempt(buf, nbytes=None):
        t = torch.from_numpy(np.frombuffer(bytes(buf), np.uint8).copy()).to(dev)
        pc.pc_decompress(t, out, ws, nbytes if nbytes is not None else len(buf))

    attempt(stream)  # the intact stream decodes
    cases = []
    b = bytearray(stream); b[0] ^= 1; cases.append((b, None))                 # magic
    b = bytearray(stream); b[4] = 2; cases.append((b, None))                  # version
    b = bytearray(stream); b[96 + 32 * 3 + 29] = 40; cases.append((b, None))  # width field > 31
    b = bytearray(stream); b[96 + 32 * 5 + 8] ^= 4; cases.append((b, None))   # word offset
    b = bytearray(stream); b[96 + 32 * 7 + 0] ^= 64; cases.append((b, None))  # particle offset
    b = bytearray(stream); b[72] ^= 8; cases.append((b, None))                # payload words
    cases.append((bytearray(stream), len(stream) - 4))                        # truncated
    # header fields the device-side validation also reads before the host has parsed them
    b = bytearray(stream); b[6] = 2; cases.append((b, None))                  # element type
    b = bytearray(stream); b[90] = 1; cases.append((b, None))                 # reserved byte
    b = bytearray(stream); b[32:40] = struct.pack("<d", float("nan")); cases.append((b, None))  # s
    b = bytearray(stream); b[64:72] = struct.pack("<Q", 60_000); cases.append((b, None))  # leaves > n
    for buf, nb in cases:
        with pytest.raises(pc.PCError) as e:
            attempt(buf, nb)
        assert e.value.status == pc.PC_ERR_CORRUPT
    # a header claiming far more particles than the workspace's chunk facts can hold: the
    # device-side validation leaves the workspace alone, the host reports the output too small
    b = bytearray(stream); b[8:16] = struct.pack("<Q", 1_000_000_000)
    with pytest.raises(pc.PCError) as e:
        attempt(b)
    assert e.value.status == pc.PC_ERR_CAPACITY
    attempt(stream)  # and the workspace still decodes the intact stream
    assert out.cpu().numpy().tobytes() == oracle_mod.decompress(stream).tobytes()
    small = torch.empty((10, 3), dtype=torch.float32, device=dev)
    with pytest.raises(pc.PCError) as e:
        pc.pc_decompress(torch.from_numpy(np.frombuffer(stream, np.uint8).copy()).to(dev), small, ws)
    assert e.value.status == pc.PC_ERR_CAPACITY


@pytest.mark.parametrize("pinned", [True, False])
@pytest.mark.parametrize("dtype", [np.float32, np.float64])
def test_host_buffer_entry_points(pc, oracle_mod, pinned, dtype):
    """Host-buffer entry points, pinned and pageable, float and double: the
    oracle's stream and positions."""
    n = 80_000
    pos = synth.cosmology(n, seed=31, dtype=dtype)
    pdt = pc.PC_F32 if dtype == np.float32 else pc.PC_F64
    pin = (lambda t: t.pin_memory()) if pinned else (lambda t: t)
    hp = pin(torch.from_numpy(pos))
    ws = torch.empty(pc.pc_compress_host_workspace_size(n, pdt), dtype=torch.uint8, device="cuda")
    hout = pin(torch.empty(pc.pc_compress_bound(n, pdt), dtype=torch.uint8))
    size = pc.pc_compress_host(hp, pc.PC_EB_REL, 1e-4, hout, ws)
    ref, _ = oracle_mod.compress(pos, oracle_mod.REL, 1e-4)
    assert hout[:size].numpy().tobytes() == ref
    dws = torch.empty(pc.pc_decompress_host_workspace_size(n, pdt, size), dtype=torch.uint8, device="cuda")
    hdec = pin(torch.empty((n, 3), dtype=hp.dtype))
    pc.pc_decompress_host(hout, size, hdec, dws)
    assert hdec.numpy().tobytes() == oracle_mod.decompress(ref).tobytes()