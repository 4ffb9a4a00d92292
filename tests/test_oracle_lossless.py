"""Pins of the oracle's lossless axes (Sec. 4.1: a dimension whose m_d exceeds M
is stored as the original coordinates, M = 32 / 64 for single / double).

Codes are at most 30 bits here (m_d <= 31), so an axis is stored losslessly when
its code range reaches 2^30, and every axis when no lattice keeps eps through
the rounding to the input type (eb' <= 0).  Pinned against what the rule and
the arithmetic fix, not against the oracle itself:
  - the coordinates of a lossless axis decode bit for bit, the other axes
    within eps;
  - the boundary of each trigger: a code range of 2^30 - 1 stays coded, 2^30
    goes lossless; eps a hair above the rounding margin stays coded, a hair
    below goes lossless;
  - the payload written bit by bit by a plain Python restatement of the
    layout (every particle, centre first; M-bit patterns; Fig. 2 codes);
  - the payload size: sum over leaves of (sum of widths) * particles;
  - the reduction and the reordering, which need codes, refuse.
"""
import math
import struct

import numpy as np
import pytest

import synth


def _bits_le(words):
    out = []
    for w in words:
        for b in range(32):
            out.append((int(w) >> b) & 1)
    return out


def _margin(pos, dtype_bits):
    """eps - eb' of Sec. 3's rounding margin, restated: ulp_T(M2) + 4 ulp_f64(M2)."""
    m = float(np.abs(pos.astype(np.float64)).max())
    m2 = 2.0 * m

    def spacing(x, prec, emin):
        e = math.frexp(x)[1] - 1
        return math.ldexp(1.0, max(e, emin) - (prec - 1))

    ut = spacing(m2, 24, -126) if dtype_bits == 32 else spacing(m2, 53, -1022)
    return ut + 4.0 * spacing(m2, 53, -1022)


@pytest.mark.parametrize("dtype,M", [(np.float32, 32), (np.float64, 64)])
def test_every_axis_lossless_below_resolution(oracle_mod, dtype, M):
    """eps below the type's spacing at the data's magnitude: all three axes
    decode bit for bit, and every leaf record carries m_d = M."""
    pos = synth.cosmology(20_000, seed=3, dtype=dtype)
    eb = 1e-9 if dtype == np.float32 else 1e-17
    b = oracle_mod.error_bound(pos, oracle_mod.REL, eb)
    assert b.raw == 7 and b.raw_cause == oracle_mod.ERR_EB_TOO_SMALL
    stream, perm = oracle_mod.compress(pos, oracle_mod.REL, eb, leaf_size=1000)
    assert stream[84] == 7
    dec = oracle_mod.decompress(stream)
    assert dec.tobytes() == pos[perm].tobytes()
    n, _, nl, _ = oracle_mod.stream_header(stream)
    for L in range(nl):
        rec = stream[96 + 32 * L: 96 + 32 * L + 32]
        assert list(rec[28:31]) == [M, M, M]
        assert struct.unpack_from("<3i", rec, 16) == (0, 0, 0)


def test_mixed_axes_wide_x(oracle_mod):
    """A slab whose x range needs codes of 2^30 or more: x losslessly, y and z as
    codes within eps."""
    rng = np.random.default_rng(1)
    pos = np.stack([rng.uniform(0, 1.0, 30_000), rng.uniform(0, 1e-6, 30_000),
                    rng.uniform(0, 2e-6, 30_000)], 1).astype(np.float64)
    eps = 1e-10
    b = oracle_mod.error_bound(pos, oracle_mod.ABS, eps)
    assert b.raw == 1 and b.raw_cause == oracle_mod.ERR_RANGE
    stream, perm = oracle_mod.compress(pos, oracle_mod.ABS, eps, leaf_size=500)
    dec = oracle_mod.decompress(stream)
    ref = pos[perm]
    assert dec[:, 0].tobytes() == ref[:, 0].tobytes()
    assert np.abs(dec[:, 1:] - ref[:, 1:]).max() <= eps
    n, _, nl, _ = oracle_mod.stream_header(stream)
    for L in range(nl):
        m = stream[96 + 32 * L + 28: 96 + 32 * L + 31]
        assert m[0] == 64 and m[1] <= 31 and m[2] <= 31


@pytest.mark.parametrize("k,raw", [((1 << 30) - 1, 0), (1 << 30, 1)])
def test_code_range_boundary(oracle_mod, k, raw):
    """x spans exactly k lattice steps: k = 2^30 - 1 keeps codes (m_x <= 31),
    k = 2^30 stores x losslessly (m_x = M = 64)."""
    eps = 1e-6
    probe = np.array([[0, 0, 0], [2100.0, 0.5, 0.5]], np.float64)  # same binade of M2 as below
    s = oracle_mod.error_bound(probe, oracle_mod.ABS, eps).s
    x = k * s
    assert 2048.0 <= x < 4096.0
    pos = np.array([[0, 0, 0], [x, 0.5, 0.5], [x / 3, 0.25, 0.1]], np.float64)
    b = oracle_mod.error_bound(pos, oracle_mod.ABS, eps)
    assert b.s == s and b.raw == raw
    stream, perm = oracle_mod.compress(pos, oracle_mod.ABS, eps, leaf_size=4)
    assert stream[84] == raw
    m_x = stream[96 + 28]
    assert (m_x == 64) if raw else (m_x <= 31)
    dec = oracle_mod.decompress(stream)
    if raw:
        assert dec[:, 0].tobytes() == pos[perm][:, 0].tobytes()
    assert np.abs(dec - pos[perm]).max() <= eps


@pytest.mark.parametrize("side,raw", [(+1, 0), (-1, 7)])
def test_rounding_margin_boundary(oracle_mod, side, raw):
    """eps a hair above Sec. 3's rounding margin keeps the lattice; a hair below,
    no lattice keeps the bound and every axis goes lossless."""
    # points a few float32 spacings apart near 1: a range small enough for
    # 30-bit codes even with a step just above zero
    rng = np.random.default_rng(2)
    pos = (1.0 + rng.integers(0, 200, (2_000, 3)) * 2.0 ** -23).astype(np.float32)
    margin = _margin(pos, 32)
    eps = margin * (1.0 + side * 1e-6)
    b = oracle_mod.error_bound(pos, oracle_mod.ABS, eps)
    assert b.raw == raw
    stream, perm = oracle_mod.compress(pos, oracle_mod.ABS, eps, leaf_size=300)
    dec = oracle_mod.decompress(stream)
    assert np.abs(dec.astype(np.float64) - pos[perm].astype(np.float64)).max() <= eps
    if raw:
        assert dec.tobytes() == pos[perm].tobytes()


@pytest.mark.parametrize("dtype", [np.float32, np.float64])
def test_payload_restated_bit_by_bit(oracle_mod, dtype):
    """The payload of a stream with lossless axes, rebuilt bit by bit in plain
    Python from the leaf table and the input: per leaf every particle, the
    centre first (its own position among the leaf's), then the rest in leaf
    order; per particle x, y, z; a lossless axis as the coordinate's M-bit
    pattern, a coded axis as (q - q_ref) + 2^(m-1) - 1 in m bits."""
    rng = np.random.default_rng(7)
    n = 700
    pos = np.stack([rng.uniform(0, 1.0, n), rng.uniform(0, 1e-5, n), rng.uniform(-1e-5, 0, n)], 1).astype(dtype)
    # float32: eps just above the rounding margin, so the step is tiny: x (range 1)
    # needs codes of 2^30 or more, y and z (range 1e-5) stay coded
    eps = 1e-10 if dtype == np.float64 else _margin(pos, 32) * 1.001
    b = oracle_mod.error_bound(pos, oracle_mod.ABS, eps)
    stream, perm = oracle_mod.compress(pos, oracle_mod.ABS, eps, leaf_size=60)
    raw = stream[84]
    assert raw == b.raw == 1
    M = 32 if dtype == np.float32 else 64
    ufmt = "<I" if M == 32 else "<Q"
    ffmt = "<f" if M == 32 else "<d"
    n_, _, nl, nw = oracle_mod.stream_header(stream)
    bits = []
    for L in range(nl):
        rec = stream[96 + 32 * L: 96 + 32 * L + 32]
        po, wo = struct.unpack_from("<QQ", rec, 0)
        qref = struct.unpack_from("<3i", rec, 16)
        m = list(rec[28:31])
        pend = struct.unpack_from("<Q", stream, 96 + 32 * (L + 1))[0] if L + 1 < nl else n
        assert len(bits) == 32 * wo
        for i in range(po, pend):  # decoded order = payload order
            p = pos[perm[i]]
            for d in range(3):
                if raw >> d & 1:
                    assert m[d] == M
                    u = struct.unpack(ufmt, struct.pack(ffmt, p[d]))[0]
                    bits += [(u >> t) & 1 for t in range(M)]
                elif m[d]:
                    # the oracle's code, recomputed: rint((p - o) / s), half to even
                    t = (float(p[d]) - b.o[d]) / b.s
                    q = int(np.rint(t))
                    c = (q - qref[d]) + (1 << (m[d] - 1)) - 1
                    assert 0 <= c <= (1 << m[d]) - 2
                    bits += [(c >> t2) & 1 for t2 in range(m[d])]
        while len(bits) % 32:
            bits.append(0)
    assert len(bits) == 32 * nw
    payload = np.frombuffer(stream, np.uint32, count=nw, offset=96 + 32 * nl)
    assert _bits_le(payload) == bits


def test_storage_term_with_lossless_axes(oracle_mod):
    """Payload words = sum over leaves of ceil((sum of widths) * particles / 32):
    every particle of a leaf, the centre included, is in the payload."""
    pos = synth.cosmology(9_000, seed=11)
    stream, _ = oracle_mod.compress(pos, oracle_mod.REL, 1e-9, leaf_size=700)
    n, _, nl, nw = oracle_mod.stream_header(stream)
    total = 0
    for L in range(nl):
        rec = stream[96 + 32 * L: 96 + 32 * L + 32]
        po = struct.unpack_from("<Q", rec, 0)[0]
        pend = struct.unpack_from("<Q", stream, 96 + 32 * (L + 1))[0] if L + 1 < nl else n
        assert struct.unpack_from("<Q", rec, 8)[0] == total
        total += (sum(rec[28:31]) * (pend - po) + 31) // 32
    assert total == nw == 3 * n  # 96 bits per float32 particle


def test_codes_refuse_lossless_axes(oracle_mod):
    """The reordering works on R-indices of codes: a stream with lossless axes is refused."""
    pos = synth.uniform(3_000, seed=5)
    stream, perm = oracle_mod.compress(pos, oracle_mod.REL, 1e-9, leaf_size=400)
    assert stream[84] == 7
    with pytest.raises(oracle_mod.OracleError) as e:
        oracle_mod.reorder(stream, perm)
    assert e.value.code == oracle_mod.ERR_ARG


def test_split_key_is_monotone_and_exact(oracle_mod):
    """The split key of a lossless axis, floor((p - lo) / (hi - lo) * 2^29),
    recomputed in Python, equals the oracle's and is monotone in p."""
    pos = synth.cosmology(5_000, seed=2)
    q = oracle_mod.quantize(pos, oracle_mod.REL, 1e-9)
    b = oracle_mod.error_bound(pos, oracle_mod.REL, 1e-9)
    for d in range(3):
        lo, hi = b.lo[d], b.hi[d]
        want = np.array([min(max(math.floor(((float(p) - lo) / (hi - lo)) * 2.0 ** 29), 0), 2 ** 29)
                         for p in pos[:, d]])
        assert np.array_equal(q[:, d], want)
        order = np.argsort(pos[:, d], kind="stable")
        assert np.all(np.diff(q[order, d]) >= 0)
    assert b.qmax == (2 ** 29, 2 ** 29, 2 ** 29)
