"""Python binding of the GB300 particle position compressor (C ABI in include/pc.h).

The functions keep the C names and only marshal arguments: torch tensors supply
device memory and streams, and every step of the compression and
decompression runs in the CUDA kernels of ``libpcbox.so``.  There is no CPU
path: if the library is missing, loading fails with an error.

Method: arXiv 2404.02826 (Ren, Di, Zhang, Zhao, Guo), error-bounded lossy
compression of particle positions with bit-adaptive quantization - lattice
quantization (Sec. 3), median k-d partition and bit boxes (Sec. 4.1, Eq. 2),
packed sequences (Sec. 4.2, Fig. 4).
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass
from typing import Optional

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libpcbox.so")

PC_OK = 0
PC_ERR_ARG = 1
PC_ERR_NONFINITE = 2
PC_ERR_EB_TOO_SMALL = 3
PC_ERR_RANGE = 4
PC_ERR_CAPACITY = 5
PC_ERR_CORRUPT = 6
PC_ERR_TIMEOUT = 7
PC_ERR_CUDA = 8
PC_F32 = 0
PC_F64 = 1
PC_EB_ABS = 0
PC_EB_REL = 1
PC_DEFAULT_LEAF_SIZE = 4096
PC_MAX_LEAF_SIZE = 12000
PC_MAX_PARTICLES = (1 << 31) - 1
PC_HEADER_BYTES = 96
PC_LEAF_BYTES = 32
PC_FLAG_AUTOTUNE_LEAF = 1
PC_FLAG_BOX_REDUCTION = 2
PC_FLAG_REORDER = 4
PC_FLAG_WIDEST_AXIS = 8
PC_FLAG_AUTOTUNE_KNOBS = 16
PC_DEFAULT_WARP_NODE_MAX = 2048
PC_MAX_WARP_NODE_MAX = 65536
PC_DEFAULT_WARP_LEAF_MAX = 1024
PC_AUTOTUNE_MIN_LEAF = 64
LEAF_AUTO = -1  # leaf_size argument: autotune with candidates up to PC_MAX_LEAF_SIZE

# every entry point declared in include/pc.h
EXPORTS = (
    "pc_compress_bound", "pc_compress_workspace_size", "pc_compress", "pc_stream_info",
    "pc_decompress_workspace_size", "pc_decompress", "pc_compress_host_workspace_size", "pc_compress_host",
    "pc_decompress_host_workspace_size", "pc_decompress_host", "pc_error_string", "pc_format_version",
    "pc_trace_enable", "pc_trace_reset", "pc_trace_count", "pc_trace_get", "pc_compress_noalloc",
    "pc_compress_batch_workspace_size", "pc_compress_batch", "pc_decompress_batch_workspace_size",
    "pc_decompress_batch", "pc_server_create", "pc_server_submit", "pc_server_poll", "pc_server_release",
    "pc_server_stats", "pc_server_destroy", "pc_server_now", "pc_leaf_size_sweep_workspace_size",
    "pc_leaf_size_sweep", "pc_selftest_wait_timeout", "pc_selftest_scatter_timeout", "pc_tuned_config",
    "pc_autotune_reset", "pc_autotune_export", "pc_autotune_import",
)
PC_REQ_COMPRESS = 0
PC_REQ_DECOMPRESS = 1
PC_NOALLOC_SCRATCH_BYTES = 48 << 20


class PCError(RuntimeError):
    def __init__(self, status: int, where: str):
        msg = _lib().pc_error_string(status).decode() if _LIB is not None else str(status)
        super().__init__(f"{where}: {msg} (status {status})")
        self.status = status


class pc_config(ctypes.Structure):
    _fields_ = [("leaf_size", ctypes.c_uint32), ("flags", ctypes.c_uint32), ("warp_node_max", ctypes.c_uint32),
                ("warp_leaf_max", ctypes.c_uint32)]


class pc_tuned_class(ctypes.Structure):
    _fields_ = [("n_bits", ctypes.c_uint32), ("dtype", ctypes.c_int32), ("device", ctypes.c_int32),
                ("flags", ctypes.c_uint32), ("leaf_size", ctypes.c_uint32), ("warp_node_max", ctypes.c_uint32),
                ("warp_leaf_max", ctypes.c_uint32), ("reserved", ctypes.c_uint32)]


class pc_info(ctypes.Structure):
    _fields_ = [("n", ctypes.c_uint64), ("dtype", ctypes.c_uint32), ("eb_mode", ctypes.c_uint32),
                ("eb", ctypes.c_double), ("eps", ctypes.c_double), ("s", ctypes.c_double),
                ("o", ctypes.c_double * 3), ("num_leaves", ctypes.c_uint64), ("payload_words", ctypes.c_uint64),
                ("leaf_size", ctypes.c_uint32), ("total_bytes", ctypes.c_uint64), ("lossless_axes", ctypes.c_uint32)]


class pc_compress_item(ctypes.Structure):
    _fields_ = [("positions", ctypes.c_void_p), ("n", ctypes.c_uint64), ("dtype", ctypes.c_int32),
                ("eb_mode", ctypes.c_int32), ("eb", ctypes.c_double), ("leaf_size", ctypes.c_uint32),
                ("flags", ctypes.c_uint32), ("out", ctypes.c_void_p), ("out_capacity", ctypes.c_uint64),
                ("out_size", ctypes.c_uint64), ("status", ctypes.c_int32), ("reserved2", ctypes.c_int32)]


class pc_decompress_item(ctypes.Structure):
    _fields_ = [("stream_data", ctypes.c_void_p), ("stream_bytes", ctypes.c_uint64), ("n", ctypes.c_uint64),
                ("out_positions", ctypes.c_void_p), ("out_capacity_bytes", ctypes.c_uint64),
                ("status", ctypes.c_int32), ("reserved", ctypes.c_int32)]


class pc_sweep_point(ctypes.Structure):
    _fields_ = [("leaf_size", ctypes.c_uint32), ("depth", ctypes.c_uint32), ("leaves", ctypes.c_uint64),
                ("header_bytes", ctypes.c_uint64), ("table_bytes", ctypes.c_uint64),
                ("payload_bytes", ctypes.c_uint64), ("total_bytes", ctypes.c_uint64)]


class pc_request(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("dtype", ctypes.c_int32), ("eb_mode", ctypes.c_int32),
                ("leaf_size", ctypes.c_uint32), ("flags", ctypes.c_uint32), ("reserved", ctypes.c_uint32),
                ("eb", ctypes.c_double), ("input", ctypes.c_void_p),
                ("n", ctypes.c_uint64), ("input_bytes", ctypes.c_uint64), ("tag", ctypes.c_uint64)]


class pc_completion(ctypes.Structure):
    _fields_ = [("tag", ctypes.c_uint64), ("status", ctypes.c_int32), ("kind", ctypes.c_int32),
                ("output", ctypes.c_void_p), ("output_bytes", ctypes.c_uint64), ("t_submit", ctypes.c_double),
                ("t_start", ctypes.c_double), ("t_done", ctypes.c_double)]


_LIB = None


def _lib():
    global _LIB
    if _LIB is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing; build it with __graft_entry__.build() "
                               "(the compressor has no CPU fallback)")
        L = ctypes.CDLL(LIB_PATH)
        u64, i32, vp, dbl = ctypes.c_uint64, ctypes.c_int, ctypes.c_void_p, ctypes.c_double
        pu64 = ctypes.POINTER(u64)
        pcfg = ctypes.POINTER(pc_config)
        L.pc_compress_bound.argtypes = [u64, i32, pcfg, pu64]
        L.pc_compress_workspace_size.argtypes = [u64, i32, pcfg, i32, pu64]
        L.pc_compress.argtypes = [vp, u64, i32, i32, dbl, pcfg, vp, u64, pu64, vp, u64, vp, vp]
        L.pc_stream_info.argtypes = [vp, u64, ctypes.POINTER(pc_info)]
        L.pc_decompress_workspace_size.argtypes = [u64, pu64]
        L.pc_decompress.argtypes = [vp, u64, vp, u64, vp, u64, vp]
        L.pc_compress_host_workspace_size.argtypes = [u64, i32, pcfg, pu64]
        L.pc_compress_host.argtypes = [vp, u64, i32, i32, dbl, pcfg, vp, u64, pu64, vp, u64, vp]
        L.pc_decompress_host_workspace_size.argtypes = [u64, i32, u64, pu64]
        L.pc_decompress_host.argtypes = [vp, u64, vp, u64, vp, u64, vp]
        L.pc_error_string.argtypes = [i32]
        L.pc_error_string.restype = ctypes.c_char_p
        L.pc_format_version.argtypes = []
        L.pc_compress_noalloc.argtypes = [vp, u64, i32, i32, dbl, pcfg, vp, u64, pu64, vp]
        L.pc_trace_enable.argtypes = [i32]
        L.pc_trace_reset.argtypes = []
        L.pc_trace_count.argtypes = []
        L.pc_trace_get.argtypes = [i32, ctypes.POINTER(ctypes.c_char_p), pu64, ctypes.POINTER(dbl)]
        u32 = ctypes.c_uint32
        L.pc_compress_batch_workspace_size.argtypes = [ctypes.POINTER(pc_compress_item), u32, u32, pu64]
        L.pc_compress_batch.argtypes = [ctypes.POINTER(pc_compress_item), u32, u32, vp, u64, vp]
        L.pc_decompress_batch_workspace_size.argtypes = [ctypes.POINTER(pc_decompress_item), u32, u32, pu64]
        L.pc_decompress_batch.argtypes = [ctypes.POINTER(pc_decompress_item), u32, u32, vp, u64, vp]
        L.pc_server_create.argtypes = [vp, u64, u32, ctypes.POINTER(vp)]
        L.pc_server_submit.argtypes = [vp, ctypes.POINTER(pc_request)]
        L.pc_server_poll.argtypes = [vp, ctypes.POINTER(pc_completion), u32, ctypes.POINTER(u32), i32]
        L.pc_server_release.argtypes = [vp, vp]
        L.pc_server_stats.argtypes = [vp, pu64, pu64]
        L.pc_server_destroy.argtypes = [vp]
        L.pc_leaf_size_sweep_workspace_size.argtypes = [u64, i32, u32, u32, pu64]
        L.pc_leaf_size_sweep.argtypes = [vp, u64, i32, i32, dbl, u32, u32, ctypes.POINTER(pc_sweep_point), u32,
                                         ctypes.POINTER(u32), vp, u64, vp]
        L.pc_server_now.argtypes = []
        L.pc_server_now.restype = dbl
        L.pc_tuned_config.argtypes = [u64, i32, pcfg, pcfg, ctypes.POINTER(i32)]
        L.pc_autotune_reset.argtypes = []
        L.pc_autotune_export.argtypes = [ctypes.POINTER(pc_tuned_class), u32, ctypes.POINTER(u32)]
        L.pc_autotune_import.argtypes = [ctypes.POINTER(pc_tuned_class), u32]
        _LIB = L
    return _LIB


def load():
    """Load the CUDA library (raises if it is not built)."""
    return _lib()


def _check(rc: int, where: str):
    if rc != PC_OK:
        raise PCError(rc, where)


def config(leaf_size: int = 0, autotune: bool = False, reduce: bool = False, reorder: bool = False,
           widest: bool = False, tune_knobs: bool = False, warp_node_max: int = 0,
           warp_leaf_max: int = 0) -> pc_config:
    """A pc_config: leaf size r (0 = default; with autotune the largest candidate,
    0 = PC_MAX_LEAF_SIZE), PC_FLAG_AUTOTUNE_LEAF, PC_FLAG_BOX_REDUCTION, PC_FLAG_REORDER,
    PC_FLAG_WIDEST_AXIS, PC_FLAG_AUTOTUNE_KNOBS, and the launch knobs (threads per node:
    warp_node_max; packing tile: warp_leaf_max; 0 = default)."""
    return pc_config(int(leaf_size), (PC_FLAG_AUTOTUNE_LEAF if autotune else 0) |
                     (PC_FLAG_BOX_REDUCTION if reduce else 0) | (PC_FLAG_REORDER if reorder else 0) |
                     (PC_FLAG_WIDEST_AXIS if widest else 0) | (PC_FLAG_AUTOTUNE_KNOBS if tune_knobs else 0),
                     int(warp_node_max), int(warp_leaf_max))


def tuned_config(n: int, dtype: int, cfg: pc_config):
    """pc_tuned_config: (the config a plain call reproduces the class's launches with, tuned?)
    for calls of (n, dtype, cfg), cfg carrying PC_FLAG_AUTOTUNE_KNOBS."""
    out = pc_config()
    tuned = ctypes.c_int(0)
    _check(_lib().pc_tuned_config(n, dtype, ctypes.byref(cfg), ctypes.byref(out), ctypes.byref(tuned)),
           "pc_tuned_config")
    return out, bool(tuned.value)


def autotune_reset() -> None:
    """pc_autotune_reset: forget every class's tuned launch knobs."""
    _check(_lib().pc_autotune_reset(), "pc_autotune_reset")


_TUNED_FIELDS = ("n_bits", "dtype", "device", "flags", "leaf_size", "warp_node_max", "warp_leaf_max")
AUTOTUNE_FORMAT = "pc-autotune-knobs"


def autotune_export() -> list:
    """pc_autotune_export: the tuned classes, as dicts of pc_tuned_class's fields."""
    L = _lib()
    count = ctypes.c_uint32(0)
    _check(L.pc_autotune_export(None, 0, ctypes.byref(count)), "pc_autotune_export")
    while True:
        arr = (pc_tuned_class * max(count.value, 1))()
        cap = count.value
        _check(L.pc_autotune_export(arr, cap, ctypes.byref(count)), "pc_autotune_export")
        if count.value <= cap:
            return [{f: int(getattr(arr[i], f)) for f in _TUNED_FIELDS} for i in range(count.value)]


def autotune_import(classes) -> None:
    """pc_autotune_import: enter classes (dicts as autotune_export gives) as tuned."""
    arr = (pc_tuned_class * max(len(classes), 1))()
    for i, c in enumerate(classes):
        for f in _TUNED_FIELDS:
            setattr(arr[i], f, int(c[f]))
    _check(_lib().pc_autotune_import(arr, len(classes)), "pc_autotune_import")


def autotune_save(path) -> int:
    """Write the tuned classes to a JSON file; returns how many."""
    import json
    classes = autotune_export()
    with open(path, "w") as f:
        json.dump({"format": AUTOTUNE_FORMAT, "version": 1, "classes": classes}, f, indent=1)
    return len(classes)


def autotune_load(path) -> int:
    """Enter the classes of a JSON file written by autotune_save as tuned; returns how many."""
    import json
    with open(path) as f:
        doc = json.load(f)
    if doc.get("format") != AUTOTUNE_FORMAT or doc.get("version") != 1:
        raise ValueError(f"{path}: not a version-1 {AUTOTUNE_FORMAT} file")
    autotune_import(doc["classes"])
    return len(doc["classes"])


def _cfg(leaf_size) -> pc_config:
    """leaf_size >= 0: that leaf size (0 = default); leaf_size < 0: autotuned
    (PC_FLAG_AUTOTUNE_LEAF) with largest candidate -leaf_size (LEAF_AUTO: the default maximum);
    a pc_config (see config()) is used as given."""
    if isinstance(leaf_size, pc_config):
        return leaf_size
    leaf_size = int(leaf_size)
    if leaf_size < 0:
        return pc_config(0 if leaf_size == LEAF_AUTO else -leaf_size, PC_FLAG_AUTOTUNE_LEAF)
    return pc_config(leaf_size, 0)


def _dtype_of(t) -> int:
    import torch
    if t.dtype == torch.float32:
        return PC_F32
    if t.dtype == torch.float64:
        return PC_F64
    raise TypeError("positions must be float32 or float64")


def _stream_handle(stream) -> int:
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return int(stream.cuda_stream)


def pc_compress_bound(n: int, dtype: int, leaf_size: int = 0) -> int:
    out = ctypes.c_uint64()
    _check(_lib().pc_compress_bound(n, dtype, ctypes.byref(_cfg(leaf_size)), ctypes.byref(out)), "pc_compress_bound")
    return out.value


def pc_compress_workspace_size(n: int, dtype: int, leaf_size: int = 0, with_perm: bool = False) -> int:
    out = ctypes.c_uint64()
    _check(_lib().pc_compress_workspace_size(n, dtype, ctypes.byref(_cfg(leaf_size)), int(with_perm),
                                             ctypes.byref(out)), "pc_compress_workspace_size")
    return out.value


def pc_compress(positions, eb_mode: int, eb: float, out, workspace, leaf_size: int = 0, perm=None,
                stream=None) -> int:
    """Compress device positions [n, 3] into the device byte tensor `out`; returns the stream size."""
    n = positions.shape[0] if positions.dim() == 2 else positions.numel() // 3
    size = ctypes.c_uint64()
    rc = _lib().pc_compress(positions.data_ptr() if n else None, n, _dtype_of(positions), eb_mode, float(eb),
                            ctypes.byref(_cfg(leaf_size)), out.data_ptr(), out.numel() * out.element_size(),
                            ctypes.byref(size), workspace.data_ptr(), workspace.numel() * workspace.element_size(),
                            perm.data_ptr() if perm is not None else None, _stream_handle(stream))
    _check(rc, "pc_compress")
    return size.value


def pc_compress_noalloc(positions, eb_mode: int, eb: float, out, leaf_size: int = 0, stream=None) -> int:
    """Compress with the library's static scratch (no device allocation by the library).

    For callers that may not allocate device memory; the scratch is a 48 MiB
    array per GPU shared by all calls, so calls must not overlap on the GPU.
    Problems that do not fit raise PCError with PC_ERR_CAPACITY."""
    n = positions.shape[0] if positions.dim() == 2 else positions.numel() // 3
    size = ctypes.c_uint64()
    rc = _lib().pc_compress_noalloc(positions.data_ptr() if n else None, n, _dtype_of(positions), eb_mode,
                                    float(eb), ctypes.byref(_cfg(leaf_size)), out.data_ptr(),
                                    out.numel() * out.element_size(), ctypes.byref(size), _stream_handle(stream))
    _check(rc, "pc_compress_noalloc")
    return size.value


@dataclass
class StreamInfo:
    n: int
    dtype: int
    eb_mode: int
    eb: float
    eps: float
    s: float
    o: tuple
    num_leaves: int
    payload_words: int
    leaf_size: int
    total_bytes: int
    lossless_axes: int = 0  # bit d: axis d stored as the original coordinates (Sec. 4.1, m_d > M)


def pc_stream_info(header: bytes) -> StreamInfo:
    info = pc_info()
    buf = ctypes.create_string_buffer(bytes(header), len(header))
    _check(_lib().pc_stream_info(buf, len(header), ctypes.byref(info)), "pc_stream_info")
    return StreamInfo(info.n, info.dtype, info.eb_mode, info.eb, info.eps, info.s, tuple(info.o), info.num_leaves,
                      info.payload_words, info.leaf_size, info.total_bytes, info.lossless_axes)


def pc_decompress_workspace_size(n: int) -> int:
    out = ctypes.c_uint64()
    _check(_lib().pc_decompress_workspace_size(n, ctypes.byref(out)), "pc_decompress_workspace_size")
    return out.value


def pc_decompress(stream_data, out_positions, workspace, nbytes: Optional[int] = None, stream=None) -> None:
    """Decompress the device byte tensor `stream_data` into device positions `out_positions`."""
    nb = nbytes if nbytes is not None else stream_data.numel()
    rc = _lib().pc_decompress(stream_data.data_ptr(), nb, out_positions.data_ptr() if out_positions.numel() else None,
                              out_positions.numel() * out_positions.element_size(), workspace.data_ptr(),
                              workspace.numel() * workspace.element_size(), _stream_handle(stream))
    _check(rc, "pc_decompress")


def pc_compress_host_workspace_size(n: int, dtype: int, leaf_size: int = 0) -> int:
    out = ctypes.c_uint64()
    _check(_lib().pc_compress_host_workspace_size(n, dtype, ctypes.byref(_cfg(leaf_size)), ctypes.byref(out)),
           "pc_compress_host_workspace_size")
    return out.value


def pc_compress_host(host_positions, eb_mode: int, eb: float, host_out, workspace, leaf_size: int = 0,
                     stream=None) -> int:
    """Host-buffer compression (CPU tensors, ideally pinned); returns the stream size."""
    n = host_positions.shape[0]
    size = ctypes.c_uint64()
    rc = _lib().pc_compress_host(host_positions.data_ptr() if n else None, n, _dtype_of(host_positions), eb_mode,
                                 float(eb), ctypes.byref(_cfg(leaf_size)), host_out.data_ptr(), host_out.numel(),
                                 ctypes.byref(size), workspace.data_ptr(), workspace.numel(), _stream_handle(stream))
    _check(rc, "pc_compress_host")
    return size.value


def pc_decompress_host_workspace_size(n: int, dtype: int, stream_bytes: int) -> int:
    out = ctypes.c_uint64()
    _check(_lib().pc_decompress_host_workspace_size(n, dtype, stream_bytes, ctypes.byref(out)),
           "pc_decompress_host_workspace_size")
    return out.value


def pc_decompress_host(host_stream, nbytes: int, host_positions, workspace, stream=None) -> None:
    rc = _lib().pc_decompress_host(host_stream.data_ptr(), nbytes, host_positions.data_ptr(),
                                   host_positions.numel() * host_positions.element_size(), workspace.data_ptr(),
                                   workspace.numel(), _stream_handle(stream))
    _check(rc, "pc_decompress_host")


def pc_selftest_wait_timeout(stream=None) -> int:
    """Runs the bounded-wait self-test; returns its status (PC_ERR_TIMEOUT when the mechanism works)."""
    L = _lib()
    L.pc_selftest_wait_timeout.argtypes = [ctypes.c_void_p]
    return int(L.pc_selftest_wait_timeout(_stream_handle(stream)))


def pc_selftest_scatter_timeout(positions, out, workspace, stream=None) -> int:
    """Runs one compress of device positions [n, 3] (n > 2^16) whose scatter tile copies
    are dropped; returns its status (PC_ERR_TIMEOUT when the failure path works)."""
    n = positions.shape[0]
    L = _lib()
    L.pc_selftest_scatter_timeout.argtypes = [ctypes.c_void_p, ctypes.c_uint64, ctypes.c_int, ctypes.c_void_p,
                                              ctypes.c_uint64, ctypes.c_void_p, ctypes.c_uint64, ctypes.c_void_p]
    return int(L.pc_selftest_scatter_timeout(positions.data_ptr(), n, _dtype_of(positions), out.data_ptr(),
                                             out.numel() * out.element_size(), workspace.data_ptr(),
                                             workspace.numel() * workspace.element_size(), _stream_handle(stream)))


def pc_error_string(status: int) -> str:
    return _lib().pc_error_string(status).decode()


def pc_format_version() -> int:
    return int(_lib().pc_format_version())


def pc_trace_enable(on: bool = True) -> None:
    _check(_lib().pc_trace_enable(int(on)), "pc_trace_enable")


def pc_trace_reset() -> None:
    _check(_lib().pc_trace_reset(), "pc_trace_reset")


def pc_trace_count() -> int:
    return int(_lib().pc_trace_count())


def pc_trace_get(i: int):
    name = ctypes.c_char_p()
    launches = ctypes.c_uint64()
    ms = ctypes.c_double()
    _check(_lib().pc_trace_get(i, ctypes.byref(name), ctypes.byref(launches), ctypes.byref(ms)), "pc_trace_get")
    return name.value.decode(), launches.value, ms.value


def trace_table() -> dict:
    """{kernel name: (launches, total ms)} accumulated while tracing was enabled."""
    return {n: (l, t) for n, l, t in (pc_trace_get(i) for i in range(pc_trace_count()))}


# ---------------------------------------------------------------------------
# convenience wrappers that take buffers from torch's allocator
# ---------------------------------------------------------------------------

def _items(cls, rows):
    arr = (cls * max(len(rows), 1))()
    for i, r in enumerate(rows):
        arr[i] = r
    return arr


def pc_compress_batch(jobs, outs, workspace=None, lanes: int = 0, stream=None):
    """Compress many device snapshots in one call.

    jobs: sequence of (positions tensor, eb_mode, eb, leaf_size); outs: device
    uint8 tensors (pc_compress_bound bytes).  Returns (stream sizes, item
    statuses); raises when the call itself fails.  The workspace (device
    uint8) is allocated here when not given."""
    import torch
    rows = []
    for (p, m, eb, leaf), o in zip(jobs, outs):
        c = _cfg(leaf)
        rows.append(pc_compress_item(p.data_ptr() if p.shape[0] else None, p.shape[0], _dtype_of(p), int(m), float(eb),
                                     c.leaf_size, c.flags, o.data_ptr(), o.numel(), 0, 0, 0))
    arr = _items(pc_compress_item, rows)
    if workspace is None:
        need = ctypes.c_uint64()
        _check(_lib().pc_compress_batch_workspace_size(arr, len(rows), lanes, ctypes.byref(need)),
               "pc_compress_batch_workspace_size")
        workspace = torch.empty(need.value, dtype=torch.uint8, device=outs[0].device if outs else "cuda")
    rc = _lib().pc_compress_batch(arr, len(rows), lanes, workspace.data_ptr(), workspace.numel(),
                                  _stream_handle(stream))
    statuses = [arr[i].status for i in range(len(rows))]
    if rc != PC_OK and all(st == PC_OK for st in statuses):
        _check(rc, "pc_compress_batch")
    return [arr[i].out_size for i in range(len(rows))], statuses


def pc_compress_batch_workspace_size(ns_dtypes_leaves, lanes: int = 0) -> int:
    """Workspace bytes for snapshots given as (n, dtype, leaf_size)."""
    rows = [pc_compress_item(None, n, dt, 0, 0.0, _cfg(leaf).leaf_size, _cfg(leaf).flags, None, 0, 0, 0, 0)
            for n, dt, leaf in ns_dtypes_leaves]
    need = ctypes.c_uint64()
    _check(_lib().pc_compress_batch_workspace_size(_items(pc_compress_item, rows), len(rows), lanes,
                                                   ctypes.byref(need)), "pc_compress_batch_workspace_size")
    return need.value


def pc_decompress_batch(streams, sizes, outs, workspace=None, lanes: int = 0, stream=None):
    """Decompress many device streams into device position tensors in one call;
    returns the item statuses."""
    import torch
    rows = []
    for st, nb, o in zip(streams, sizes, outs):
        rows.append(pc_decompress_item(st.data_ptr(), int(nb), o.shape[0], o.data_ptr(),
                                       o.numel() * o.element_size(), 0, 0))
    arr = _items(pc_decompress_item, rows)
    if workspace is None:
        need = ctypes.c_uint64()
        _check(_lib().pc_decompress_batch_workspace_size(arr, len(rows), lanes, ctypes.byref(need)),
               "pc_decompress_batch_workspace_size")
        workspace = torch.empty(need.value, dtype=torch.uint8, device=outs[0].device if outs else "cuda")
    rc = _lib().pc_decompress_batch(arr, len(rows), lanes, workspace.data_ptr(), workspace.numel(),
                                    _stream_handle(stream))
    statuses = [arr[i].status for i in range(len(rows))]
    if rc != PC_OK and all(st == PC_OK for st in statuses):
        _check(rc, "pc_decompress_batch")
    return statuses


def pc_leaf_size_sweep(positions, eb_mode: int, eb: float, r_min: int = 1024, r_max: int = PC_MAX_LEAF_SIZE,
                       workspace=None, stream=None):
    """Stream size and parts for every candidate leaf size ceil(n / 2^d) in [r_min, r_max], largest first."""
    import torch
    n = positions.shape[0]
    dt = _dtype_of(positions)
    if workspace is None:
        need = ctypes.c_uint64()
        _check(_lib().pc_leaf_size_sweep_workspace_size(n, dt, r_min, r_max, ctypes.byref(need)),
               "pc_leaf_size_sweep_workspace_size")
        workspace = torch.empty(max(need.value, 1), dtype=torch.uint8, device=positions.device)
    pts = (pc_sweep_point * 64)()
    cnt = ctypes.c_uint32()
    _check(_lib().pc_leaf_size_sweep(positions.data_ptr() if n else None, n, dt, int(eb_mode), float(eb), int(r_min),
                                     int(r_max), pts, 64, ctypes.byref(cnt), workspace.data_ptr(), workspace.numel(),
                                     _stream_handle(stream)), "pc_leaf_size_sweep")
    return [{f: getattr(pts[i], f) for f, _ in pc_sweep_point._fields_} for i in range(min(cnt.value, 64))]


class Server:
    """The serving loop of the library (pc_server_*): worker lanes admit queued
    requests into a device arena as room frees up; outputs stay in the arena
    until released."""

    def __init__(self, arena, lanes: int = 4):
        self.arena = arena  # device uint8 tensor, kept alive here
        h = ctypes.c_void_p()
        _check(_lib().pc_server_create(arena.data_ptr(), arena.numel(), lanes, ctypes.byref(h)), "pc_server_create")
        self.h = h

    def submit_compress(self, positions, eb_mode: int, eb: float, tag: int, leaf_size: int = 0):
        c = _cfg(leaf_size)
        r = pc_request(PC_REQ_COMPRESS, _dtype_of(positions), int(eb_mode), c.leaf_size, c.flags, 0, float(eb),
                       positions.data_ptr(), positions.shape[0], 0, int(tag))
        _check(_lib().pc_server_submit(self.h, ctypes.byref(r)), "pc_server_submit")

    def submit_decompress(self, stream_data, nbytes: int, n: int, dtype: int, tag: int):
        r = pc_request(PC_REQ_DECOMPRESS, int(dtype), 0, 0, 0, 0, 0.0, stream_data.data_ptr(), int(n), int(nbytes),
                       int(tag))
        _check(_lib().pc_server_submit(self.h, ctypes.byref(r)), "pc_server_submit")

    def poll(self, wait: bool = False, max_items: int = 256):
        buf = (pc_completion * max_items)()
        got = ctypes.c_uint32()
        _check(_lib().pc_server_poll(self.h, buf, max_items, ctypes.byref(got), 1 if wait else 0), "pc_server_poll")
        return [buf[i] for i in range(got.value)]

    def output(self, c, dtype=None):
        """A view of a completion's output in the arena (uint8, or positions [n, 3] given dtype)."""
        import torch
        off = c.output - self.arena.data_ptr()
        v = self.arena[off: off + c.output_bytes]
        return v if dtype is None else v.view(dtype).view(-1, 3)

    def release(self, c):
        _check(_lib().pc_server_release(self.h, c.output), "pc_server_release")

    def stats(self):
        p, u = ctypes.c_uint64(), ctypes.c_uint64()
        _check(_lib().pc_server_stats(self.h, ctypes.byref(p), ctypes.byref(u)), "pc_server_stats")
        return p.value, u.value

    def close(self):
        if self.h:
            _check(_lib().pc_server_destroy(self.h), "pc_server_destroy")
            self.h = None

    @staticmethod
    def now() -> float:
        return _lib().pc_server_now()


class Compressor:
    """Holds device buffers sized for one problem size and reuses them."""

    def __init__(self, n: int, dtype: int, leaf_size: int = 0, with_perm: bool = False, device="cuda"):
        import torch
        self.n, self.dtype, self.leaf_size, self.with_perm = n, dtype, leaf_size, with_perm
        self.out = torch.empty(pc_compress_bound(n, dtype, leaf_size), dtype=torch.uint8, device=device)
        self.ws = torch.empty(pc_compress_workspace_size(n, dtype, leaf_size, with_perm), dtype=torch.uint8,
                              device=device)
        self.perm = torch.empty(max(n, 1), dtype=torch.int32, device=device) if with_perm else None
        self.dws = torch.empty(pc_decompress_workspace_size(n), dtype=torch.uint8, device=device)

    def compress(self, positions, eb_mode: int, eb: float, stream=None) -> int:
        return pc_compress(positions, eb_mode, eb, self.out, self.ws, self.leaf_size, self.perm, stream)

    def decompress(self, stream_data, out_positions, nbytes=None, stream=None) -> None:
        pc_decompress(stream_data, out_positions, self.dws, nbytes, stream)


def compress(positions, eb_mode: int, eb: float, leaf_size: int = 0, with_perm: bool = False):
    """One-shot compression; returns (stream tensor on the device, perm or None)."""
    n = positions.shape[0]
    c = Compressor(n, _dtype_of(positions), leaf_size, with_perm, positions.device)
    size = c.compress(positions, eb_mode, eb)
    return c.out[:size].clone(), (c.perm[:n].clone() if with_perm else None)


def decompress(stream_data):
    """One-shot decompression of a device stream tensor; returns positions [n, 3] on the device."""
    import torch
    info = pc_stream_info(stream_data[:PC_HEADER_BYTES].cpu().numpy().tobytes())
    dt = torch.float32 if info.dtype == PC_F32 else torch.float64
    out = torch.empty((info.n, 3), dtype=dt, device=stream_data.device)
    ws = torch.empty(pc_decompress_workspace_size(info.n), dtype=torch.uint8, device=stream_data.device)
    pc_decompress(stream_data, out, ws, info.total_bytes)
    return out
