"""A third, pure-Python reader of the compressed stream, for tests.

It parses the header, the per-sequence table and the packed codes without
touching either implementation, so that tests can inspect widths, centres and
codes of streams written by the oracle or by the CUDA library.

Layout (Sec. 4.2 / Fig. 4 of arXiv 2404.02826, adapted: the centre is stored
as its lattice code and an explicit particle count replaces the end mark):
  header, 96 bytes: "PCB1", u16 version, u8 dtype, u8 eb_mode, u64 n,
      f64 eb, f64 eps, f64 s, f64 o[3], u64 num_leaves, u64 payload_words,
      u32 leaf_size, 12 zero bytes;
  leaf table, 32 bytes per leaf: u64 first particle, u64 first word,
      i32 q_ref[3], u8 m[3], u8 zero;
  payload: u32 words; per leaf, the non-centre particles in leaf order, each
      as c_x (m_x bits), c_y, c_z, least-significant bit first.
"""
from __future__ import annotations

import struct
from dataclasses import dataclass, field

import numpy as np

HEADER = 96
LEAF = 32


@dataclass
class Leaf:
    particle_offset: int
    word_offset: int
    q_ref: tuple
    m: tuple
    count: int = 0
    codes: list = field(default_factory=list)


@dataclass
class Stream:
    version: int
    dtype: int
    eb_mode: int
    n: int
    eb: float
    eps: float
    s: float
    o: tuple
    num_leaves: int
    payload_words: int
    leaf_size: int
    leaves: list
    words: np.ndarray


def parse(buf: bytes, with_codes: bool = True) -> Stream:
    buf = bytes(buf)
    assert buf[:4] == b"PCB1", "bad magic"
    version, dtype, eb_mode, n = struct.unpack_from("<HBBQ", buf, 4)
    eb, eps, s, ox, oy, oz = struct.unpack_from("<6d", buf, 16)
    num_leaves, payload_words, leaf_size = struct.unpack_from("<QQI", buf, 64)
    assert buf[84:96] == b"\0" * 12
    leaves = []
    for L in range(num_leaves):
        po, wo, qx, qy, qz, mx, my, mz, z = struct.unpack_from("<QQiii4B", buf, HEADER + LEAF * L)
        assert z == 0
        leaves.append(Leaf(po, wo, (qx, qy, qz), (mx, my, mz)))
    for L in range(num_leaves):
        end = leaves[L + 1].particle_offset if L + 1 < num_leaves else n
        leaves[L].count = end - leaves[L].particle_offset
    start = HEADER + LEAF * num_leaves
    words = np.frombuffer(buf, dtype="<u4", count=payload_words, offset=start).copy()
    st = Stream(version, dtype, eb_mode, n, eb, eps, s, (ox, oy, oz), num_leaves, payload_words, leaf_size, leaves,
                words)
    if with_codes:
        big = int.from_bytes(words.tobytes(), "little")
        for lf in leaves:
            pos = 32 * lf.word_offset
            for _ in range(lf.count - 1):
                c = []
                for d in range(3):
                    md = lf.m[d]
                    c.append((big >> pos) & ((1 << md) - 1) if md else 0)
                    pos += md
                lf.codes.append(tuple(c))
    return st


def decoded_codes(st: Stream) -> np.ndarray:
    """Lattice codes of every decoded particle, in stream order (centre first per leaf)."""
    out = []
    for lf in st.leaves:
        out.append(lf.q_ref)
        for c in lf.codes:
            out.append(tuple(lf.q_ref[d] + c[d] - ((1 << (lf.m[d] - 1)) - 1) if lf.m[d] else lf.q_ref[d]
                             for d in range(3)))
    return np.asarray(out, dtype=np.int64).reshape(-1, 3)
