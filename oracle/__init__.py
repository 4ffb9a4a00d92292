"""Python access to the CPU oracle (``oracle/oracle.c``).

TEST INFRASTRUCTURE ONLY.  The oracle is a plain, slow, double-precision CPU
restatement of the bit-adaptive particle compressor (arXiv 2404.02826: Sec. 3
error bound and quantization, Sec. 4.1 k-d partition and bit boxes, Eq. 2,
Sec. 4.2 / Fig. 4 sequence layout, Sec. 5.1 metrics).  Only ``tests/``,
``__graft_entry__.smoke()`` and the CPU-baseline legs of ``bench.py`` import
this module; the CUDA library never does, and this module imports nothing
from it.

Functions without a pin other than the ones listed in the test suite:
the compression ratio has no value in the paper that is comparable to this
stream (parity unpinned beyond the storage-cost bit count of Sec. 4.2).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "_liboracle.so")
_LIB_OMP = os.path.join(_HERE, "_liboracle_omp.so")  # the same source built with -fopenmp

OK, ERR_ARG, ERR_NONFINITE, ERR_EB_TOO_SMALL, ERR_RANGE, ERR_CAPACITY, ERR_CORRUPT = range(7)
F32, F64 = 0, 1
ABS, REL = 0, 1


class OracleError(RuntimeError):
    def __init__(self, code: int, what: str):
        super().__init__(f"{what}: oracle status {code}")
        self.code = code


def build(force: bool = False, parallel: bool = False) -> str:
    """Compile the oracle with gcc (-O2, no floating-point contraction); with
    parallel=True the same source with -fopenmp."""
    target = _LIB_OMP if parallel else _LIB
    if not force and os.path.exists(target) and os.path.getmtime(target) >= os.path.getmtime(_SRC):
        return target
    tmp = target + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared"] + \
          (["-fopenmp"] if parallel else []) + ["-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, target)
    return target


class _Bound(ctypes.Structure):
    _fields_ = [("lo", ctypes.c_double * 3), ("hi", ctypes.c_double * 3), ("delta_max", ctypes.c_double),
                ("eps", ctypes.c_double), ("eb_prime", ctypes.c_double), ("s", ctypes.c_double),
                ("o", ctypes.c_double * 3), ("qmax", ctypes.c_int64 * 3), ("raw", ctypes.c_uint32),
                ("raw_cause", ctypes.c_int)]


_libs = {}


def lib(parallel: bool = False):
    """The oracle library; parallel=True loads the OpenMP build of the same source."""
    if parallel not in _libs:
        L = ctypes.CDLL(build(parallel=parallel))
        u64, i32, dbl, vp = ctypes.c_uint64, ctypes.c_int, ctypes.c_double, ctypes.c_void_p
        L.oracle_error_bound.argtypes = [vp, u64, i32, i32, dbl, ctypes.POINTER(_Bound)]
        L.oracle_quantize.argtypes = [vp, u64, i32, ctypes.POINTER(_Bound), vp]
        L.oracle_kdtree.argtypes = [vp, u64, u64, vp, ctypes.POINTER(vp), ctypes.POINTER(vp),
                                    ctypes.POINTER(u64)]
        L.oracle_kdtree_rule.argtypes = [vp, u64, u64, i32, vp, ctypes.POINTER(vp), ctypes.POINTER(vp),
                                         ctypes.POINTER(u64)]
        L.oracle_compress_rule.argtypes = [vp, u64, i32, i32, dbl, u64, i32, ctypes.POINTER(vp), ctypes.POINTER(u64),
                                           ctypes.POINTER(vp)]
        L.oracle_num_bits.argtypes = [u64]
        L.oracle_num_bits.restype = ctypes.c_uint32
        L.oracle_bitbox.argtypes = [vp, u64, ctypes.POINTER(u64), vp, vp, vp, vp]
        L.oracle_compress.argtypes = [vp, u64, i32, i32, dbl, u64, ctypes.POINTER(vp), ctypes.POINTER(u64),
                                      ctypes.POINTER(vp)]
        L.oracle_compress_reduced.argtypes = [vp, u64, i32, i32, dbl, u64, i32, i32, ctypes.POINTER(vp),
                                              ctypes.POINTER(u64),
                                              ctypes.POINTER(vp), ctypes.POINTER(u64)]
        L.oracle_reorder.argtypes = [vp, u64, vp, ctypes.POINTER(vp), ctypes.POINTER(u64), vp, vp]
        L.oracle_rindex.argtypes = [vp, vp, vp, ctypes.POINTER(u64), ctypes.POINTER(u64)]
        L.oracle_rindex.restype = None
        L.oracle_axis_order.argtypes = [vp, u64, vp, vp]
        L.oracle_axis_order.restype = None
        L.oracle_stream_header.argtypes = [vp, u64, ctypes.POINTER(u64), ctypes.POINTER(i32),
                                           ctypes.POINTER(u64), ctypes.POINTER(u64)]
        L.oracle_decompress.argtypes = [vp, u64, vp, u64]
        L.oracle_nrmse.argtypes = [vp, vp, vp, u64, i32, dbl]
        L.oracle_nrmse.restype = dbl
        L.oracle_psnr.argtypes = [dbl]
        L.oracle_psnr.restype = dbl
        L.oracle_num_leaves.argtypes = [u64, u64]
        L.oracle_num_leaves.restype = u64
        L.oracle_free.argtypes = [vp]
        _libs[parallel] = L
    return _libs[parallel]


def _dtype_code(arr: np.ndarray) -> int:
    if arr.dtype == np.float32:
        return F32
    if arr.dtype == np.float64:
        return F64
    raise TypeError("positions must be float32 or float64")


def _positions(pos) -> np.ndarray:
    pos = np.ascontiguousarray(pos)
    if pos.ndim != 2 or pos.shape[1] != 3:
        pos = pos.reshape(-1, 3)
    return pos


@dataclass
class Bound:
    lo: tuple
    hi: tuple
    delta_max: float
    eps: float
    eb_prime: float
    s: float
    o: tuple
    qmax: tuple
    raw: int = 0        # bit d: axis d stored losslessly (Sec. 4.1, m_d > M)
    raw_cause: int = 0  # EB_TOO_SMALL (no lattice meets eps) or RANGE (codes of 2^30 or more)


def error_bound(pos, eb_mode: int, eb: float) -> Bound:
    """Sec. 3: eps from the absolute or value-range-relative bound, the lattice step and origin."""
    pos = _positions(pos)
    b = _Bound()
    rc = lib().oracle_error_bound(pos.ctypes.data if pos.size else None, pos.shape[0], _dtype_code(pos),
                                  eb_mode, float(eb), ctypes.byref(b))
    if rc:
        raise OracleError(rc, "error_bound")
    return Bound(tuple(b.lo), tuple(b.hi), b.delta_max, b.eps, b.eb_prime, b.s, tuple(b.o), tuple(b.qmax), b.raw,
                 b.raw_cause)


def quantize(pos, eb_mode: int, eb: float) -> np.ndarray:
    """Sec. 3: lattice codes q[n, 3] (int64); on an axis stored losslessly, its split key."""
    pos = _positions(pos)
    b = error_bound(pos, eb_mode, eb)
    cb = _Bound()
    cb.o[:] = b.o
    cb.s = b.s
    cb.lo[:] = b.lo
    cb.hi[:] = b.hi
    cb.raw = b.raw
    q = np.zeros((pos.shape[0], 3), np.int64)
    lib().oracle_quantize(pos.ctypes.data if pos.size else None, pos.shape[0], _dtype_code(pos),
                          ctypes.byref(cb), q.ctypes.data)
    return q


def kdtree(q: np.ndarray, leaf_size: int, widest: bool = False):
    """Sec. 4.1: returns (order, leaf_off, leaf_cnt); order lists original indices leaf by leaf.
    widest: split each node on the axis of its widest cell instead of depth mod 3."""
    q = np.ascontiguousarray(q, dtype=np.int64).reshape(-1, 3)
    n = q.shape[0]
    order = np.zeros(max(n, 1), np.uint64)
    po, pc = ctypes.c_void_p(), ctypes.c_void_p()
    nl = ctypes.c_uint64()
    rc = lib().oracle_kdtree_rule(q.ctypes.data, n, leaf_size, int(widest), order.ctypes.data, ctypes.byref(po),
                                  ctypes.byref(pc), ctypes.byref(nl))
    if rc:
        raise OracleError(rc, "kdtree")
    k = nl.value
    off = np.ctypeslib.as_array(ctypes.cast(po, ctypes.POINTER(ctypes.c_uint64)), (k,)).copy() if k else \
        np.zeros(0, np.uint64)
    cnt = np.ctypeslib.as_array(ctypes.cast(pc, ctypes.POINTER(ctypes.c_uint64)), (k,)).copy() if k else \
        np.zeros(0, np.uint64)
    lib().oracle_free(po)
    lib().oracle_free(pc)
    return order[:n].astype(np.int64), off.astype(np.int64), cnt.astype(np.int64)


def num_bits(R: int) -> int:
    """Eq. 2 on the lattice: bits for a largest centre distance of R lattice steps."""
    return int(lib().oracle_num_bits(int(R)))


def quantize_on(pos, o, s: float) -> np.ndarray:
    """Sec. 3: lattice codes q[n, 3] (int64) on a given lattice (origin o, step s)."""
    pos = _positions(pos)
    cb = _Bound()
    cb.o[:] = tuple(float(x) for x in o)
    cb.s = float(s)
    q = np.zeros((pos.shape[0], 3), np.int64)
    lib().oracle_quantize(pos.ctypes.data if pos.size else None, pos.shape[0], _dtype_code(pos), ctypes.byref(cb),
                          q.ctypes.data)
    return q


def bitbox(leafq: np.ndarray):
    """Sec. 4.1: (centre position, lo[3], hi[3], q_ref[3], m[3]) of one leaf."""
    leafq = np.ascontiguousarray(leafq, dtype=np.int64).reshape(-1, 3)
    c = ctypes.c_uint64()
    lo, hi, qref = (np.zeros(3, np.int64) for _ in range(3))
    m = np.zeros(3, np.uint32)
    rc = lib().oracle_bitbox(leafq.ctypes.data, leafq.shape[0], ctypes.byref(c), lo.ctypes.data, hi.ctypes.data,
                             qref.ctypes.data, m.ctypes.data)
    if rc:
        raise OracleError(rc, "bitbox")
    return int(c.value), lo, hi, qref, m.astype(np.int64)


def compress(pos, eb_mode: int, eb: float, leaf_size: int = 4096, want_perm: bool = True, parallel: bool = False,
             widest: bool = False):
    """Full compression.  Returns (stream bytes, perm) with perm[decoded i] = original index.
    widest: split each node on the axis of its widest cell instead of depth mod 3."""
    pos = _positions(pos)
    out = ctypes.c_void_p()
    nbytes = ctypes.c_uint64()
    perm = ctypes.c_void_p()
    L = lib(parallel)
    rc = L.oracle_compress_rule(pos.ctypes.data if pos.size else None, pos.shape[0], _dtype_code(pos), eb_mode,
                                float(eb), leaf_size, int(widest), ctypes.byref(out), ctypes.byref(nbytes),
                                ctypes.byref(perm) if want_perm else None)
    if rc:
        raise OracleError(rc, "compress")
    stream = ctypes.string_at(out, nbytes.value)
    L.oracle_free(out)
    p = None
    if want_perm:
        n = pos.shape[0]
        p = np.ctypeslib.as_array(ctypes.cast(perm, ctypes.POINTER(ctypes.c_uint64)), (n,)).astype(np.int64) \
            if n else np.zeros(0, np.int64)
        L.oracle_free(perm)
    return stream, p


def compress_reduced(pos, eb_mode: int, eb: float, leaf_size: int = 4096, want_perm: bool = True,
                     parallel: bool = False, one_per_round: bool = False, widest: bool = False):
    """Compression with the bit-box reduction in rounds (Sec. 4.1, Alg. 1; see oracle.c).
    one_per_round removes a single box (the smallest key) per round, the paper's order.
    Returns (stream bytes, perm, rounds)."""
    pos = _positions(pos)
    out = ctypes.c_void_p()
    nbytes = ctypes.c_uint64()
    perm = ctypes.c_void_p()
    rounds = ctypes.c_uint64()
    L = lib(parallel)
    rc = L.oracle_compress_reduced(pos.ctypes.data if pos.size else None, pos.shape[0], _dtype_code(pos), eb_mode,
                                   float(eb), leaf_size, int(widest), int(one_per_round), ctypes.byref(out),
                                   ctypes.byref(nbytes),
                                   ctypes.byref(perm) if want_perm else None, ctypes.byref(rounds))
    if rc:
        raise OracleError(rc, "compress_reduced")
    stream = ctypes.string_at(out, nbytes.value)
    L.oracle_free(out)
    p = None
    if want_perm:
        n = pos.shape[0]
        p = np.ctypeslib.as_array(ctypes.cast(perm, ctypes.POINTER(ctypes.c_uint64)), (n,)).astype(np.int64) \
            if n else np.zeros(0, np.int64)
        L.oracle_free(perm)
    return stream, p, rounds.value


def rindex(c, m, order) -> int:
    """Sec. 4.2: the R-index of codes c[3] of widths m[3], axes in `order` (most significant first)."""
    cc = np.asarray(c, np.uint32)
    mm = np.asarray(m, np.uint32)
    oo = np.asarray(order, np.int32)
    hi, lo = ctypes.c_uint64(), ctypes.c_uint64()
    lib().oracle_rindex(cc.ctypes.data, mm.ctypes.data, oo.ctypes.data, ctypes.byref(hi), ctypes.byref(lo))
    return (hi.value << 64) | lo.value


def axis_order(m):
    """Sec. 4.2: axes in increasing entropy of their m_d over sequences (m: k x 3). Returns (order, entropies)."""
    mm = np.ascontiguousarray(m, np.uint32).reshape(-1, 3)
    order = np.zeros(3, np.int32)
    ent = np.zeros(3, np.float64)
    lib().oracle_axis_order(mm.ctypes.data, mm.shape[0], order.ctypes.data, ent.ctypes.data)
    return tuple(int(x) for x in order), ent


def reorder(stream: bytes, perm=None):
    """Sec. 4.2 reordering of a stream: sequences by sum m_d, particles by R-index.
    Returns (stream, perm, axis order); perm maps new positions to input indices
    (to the old positions when perm is None)."""
    n, _, _, _ = stream_header(stream)
    buf = ctypes.create_string_buffer(bytes(stream), len(stream))
    pin = None if perm is None else np.ascontiguousarray(perm, np.uint64)
    pout = np.zeros(max(n, 1), np.uint64)
    order = np.zeros(3, np.int32)
    out = ctypes.c_void_p()
    nbytes = ctypes.c_uint64()
    rc = lib().oracle_reorder(buf, len(stream), None if pin is None else pin.ctypes.data, ctypes.byref(out),
                              ctypes.byref(nbytes), pout.ctypes.data, order.ctypes.data)
    if rc:
        raise OracleError(rc, "reorder")
    res = ctypes.string_at(out, nbytes.value)
    lib().oracle_free(out)
    return res, pout[:n].astype(np.int64), tuple(int(x) for x in order)


def stream_header(stream: bytes):
    n, nl, nw = ctypes.c_uint64(), ctypes.c_uint64(), ctypes.c_uint64()
    dt = ctypes.c_int()
    buf = ctypes.create_string_buffer(stream, len(stream))
    rc = lib().oracle_stream_header(buf, len(stream), ctypes.byref(n), ctypes.byref(dt), ctypes.byref(nl),
                                    ctypes.byref(nw))
    if rc:
        raise OracleError(rc, "stream_header")
    return n.value, dt.value, nl.value, nw.value


def decompress(stream: bytes, parallel: bool = False) -> np.ndarray:
    """Sec. 3 dequantization of every sequence; returns positions [n, 3] in stream order."""
    n, dt, _, _ = stream_header(stream)
    out = np.zeros((n, 3), np.float32 if dt == F32 else np.float64)
    buf = ctypes.create_string_buffer(stream, len(stream))
    rc = lib(parallel).oracle_decompress(buf, len(stream), out.ctypes.data if n else None, out.nbytes)
    if rc:
        raise OracleError(rc, "decompress")
    return out


def nrmse(orig, dec, perm, delta_max: float) -> float:
    """Sec. 5.1 NRMSE over particles matched through perm."""
    orig = _positions(orig)
    dec = _positions(dec)
    perm = np.ascontiguousarray(perm, dtype=np.uint64)
    return float(lib().oracle_nrmse(orig.ctypes.data, dec.ctypes.data, perm.ctypes.data, orig.shape[0],
                                    _dtype_code(orig), delta_max))


def psnr(nrmse_value: float) -> float:
    """Sec. 5.1: PSNR = -20 log10 NRMSE."""
    return float(lib().oracle_psnr(nrmse_value))


def num_leaves(n: int, leaf_size: int) -> int:
    return int(lib().oracle_num_leaves(n, leaf_size))
