"""Thin ctypes binding of the C ABI in ``include/olap.h``.

Argument marshalling only: every step of the offloaded path runs in the CUDA
library ``_build/libolap.so``.  Loading fails loudly when that library is
missing; there is no CPU fallback.  Buffers may be numpy arrays (pageable host
memory), pinned CPU torch tensors or CUDA torch tensors; the memory kind is
derived from the object and passed through the ABI.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

from . import build as _build

# Status codes (olap_status)
OK, E_INVALID, E_NOMEM, E_CUDA, E_OVERFLOW, E_TIMEOUT, E_UNIMPLEMENTED, E_DEVICE = range(8)
STATUS_NAMES = ["OK", "E_INVALID", "E_NOMEM", "E_CUDA", "E_OVERFLOW", "E_TIMEOUT",
                "E_UNIMPLEMENTED", "E_DEVICE"]
KEY_I64, KEY_F32, KEY_F64, KEY_U64, KEY_I32, KEY_U32 = 0, 1, 2, 3, 4, 5
KEY_NUMPY = {KEY_I64: np.int64, KEY_F32: np.float32, KEY_F64: np.float64, KEY_U64: np.uint64,
             KEY_I32: np.int32, KEY_U32: np.uint32}
ASC, DESC = 0, 1
MEM_HOST, MEM_HOST_PINNED, MEM_DEVICE = 0, 1, 2

# Every symbol include/olap.h declares, checked by the ABI tests.
EXPORTS = [
    "olap_ctx_create", "olap_ctx_destroy", "olap_last_error", "olap_ctx_stream", "olap_ctx_sync",
    "olap_ctx_host_direct", "olap_selftest_wait",
    "olap_topk", "olap_topk_pair", "olap_topk_async", "olap_topk_noalloc", "olap_topk_info_last", "olap_topk_rows",
    "olap_ctx_time_kernels", "olap_kernel_ms_last", "olap_ctx_launches", "olap_autotune",
    "olap_join_build", "olap_join_probe", "olap_join_probe_async", "olap_join_probe_partitions",
    "olap_join_probe_info_last",
    "olap_join_table_info", "olap_join_free",
    "olap_gate_calibrate", "olap_gate_estimate",
    "olap_batch_create", "olap_batch_run", "olap_batch_run_per_query", "olap_batch_errors", "olap_batch_free",
    "olap_serve",
]
SERVE_GATED, SERVE_ALWAYS_GPU, SERVE_ALWAYS_HOST = 0, 1, 2
OP_TOPK, OP_PROBE = 0, 1
CPU_NLOGN, CPU_NK, CPU_NM, CPU_MAX = 0, 1, 2, 3
FIT_ORDINARY, FIT_RELATIVE = 0, 1
FILTER_AUTO, FILTER_BULK, FILTER_REGS = 0, 1, 2
LOADS_AUTO, LOADS_L1, LOADS_L2_ONLY = 0, 1, 2
HOST_AUTO, HOST_STAGED = 0, 1
PREFILTER_AUTO, PREFILTER_OFF, PREFILTER_ON = 0, 1, 2
NOALLOC_MAX_N = 1 << 24
NOALLOC_MAX_K = 4096


class OlapError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES[status] if 0 <= status < len(STATUS_NAMES) else status}: {msg}")
        self.status = status


class olap_opts(ctypes.Structure):
    _fields_ = [
        ("device", ctypes.c_int),
        ("stream", ctypes.c_void_p),
        ("mem_budget_bytes", ctypes.c_uint64),
        ("margin_ms", ctypes.c_double),
        ("block_threads", ctypes.c_int),
        ("load_factor", ctypes.c_double),
        ("staging_bytes", ctypes.c_uint64),
        ("topk_filter", ctypes.c_int),
        ("topk_tile_bytes", ctypes.c_int),
        ("topk_stages", ctypes.c_int),
        ("topk_ctas_per_sm", ctypes.c_int),
        ("join_partitions", ctypes.c_int),
        ("join_bucket_loads", ctypes.c_int),
        ("l2_fetch_bytes", ctypes.c_int),
        ("topk_digit_bits", ctypes.c_int),
        ("host_access", ctypes.c_int),
        ("batch_overlap", ctypes.c_int),
        ("batch_topk_ctas_per_sm", ctypes.c_int),
        ("join_prefilter", ctypes.c_int),
        ("staging_threads", ctypes.c_int),
    ]


_dp = ctypes.POINTER(ctypes.c_double)


class olap_gate_samples(ctypes.Structure):
    _fields_ = [("op", ctypes.c_int), ("weighting", ctypes.c_int), ("count", ctypes.c_uint64), ("n", _dp),
                ("k_or_m", _dp),
                ("tx_bytes", _dp), ("out_rows", _dp), ("t_cpu_ms", _dp), ("t_tx_ms", _dp),
                ("t_ker_ms", _dp), ("t_post_ms", _dp), ("topk_cpu", ctypes.c_int), ("pad", ctypes.c_int),
                ("cpu_split_n", ctypes.c_double)]


class olap_gate_model(ctypes.Structure):
    _fields_ = [("op", ctypes.c_int), ("cpu_form", ctypes.c_int)] + \
        [(nm, ctypes.c_double) for nm in ("a", "b", "c", "d", "e", "f", "g", "h", "margin_ms", "rss_nlogn",
                                          "rss_nk", "a2", "b2", "split_n", "a_hi", "b_hi", "a2_hi", "b2_hi")]


class olap_gate_query(ctypes.Structure):
    _fields_ = [("op", ctypes.c_int), ("n", ctypes.c_uint64), ("k_or_m", ctypes.c_double),
                ("tx_bytes", ctypes.c_double), ("out_rows", ctypes.c_double),
                ("bytes_per_row", ctypes.c_double), ("out_per_row", ctypes.c_double)]


class olap_gate_decision(ctypes.Structure):
    _fields_ = [("offload", ctypes.c_int)] + \
        [(nm, ctypes.c_double) for nm in ("c_cpu", "c_tx", "c_ker", "c_post", "c_gpu", "gain_ms", "margin_ms")] + \
        [("n_star", ctypes.c_uint64)]


class olap_batch_item(ctypes.Structure):
    _fields_ = [("op", ctypes.c_int), ("key_type", ctypes.c_int), ("order", ctypes.c_int),
                ("keys", ctypes.c_void_p), ("rowids", ctypes.c_void_p), ("n", ctypes.c_uint64),
                ("k", ctypes.c_uint64), ("out_keys", ctypes.c_void_p), ("out_rowids", ctypes.c_void_p),
                ("table", ctypes.c_void_p), ("out_pairs", ctypes.c_void_p), ("capacity", ctypes.c_uint64),
                ("count", ctypes.c_void_p), ("status", ctypes.c_void_p)]


class olap_serve_request(ctypes.Structure):
    _fields_ = [("op", ctypes.c_int), ("key_type", ctypes.c_int), ("order", ctypes.c_int), ("table_id", ctypes.c_int),
                ("keys", ctypes.c_void_p), ("rowids", ctypes.c_void_p), ("n", ctypes.c_uint64), ("k", ctypes.c_uint64),
                ("table", ctypes.c_void_p), ("expected_pairs", ctypes.c_double), ("arrival_ms", ctypes.c_double),
                ("out_keys", ctypes.c_void_p), ("out_rowids", ctypes.c_void_p), ("out_pairs", ctypes.c_void_p),
                ("capacity", ctypes.c_uint64), ("out_count", ctypes.c_uint64), ("status", ctypes.c_int),
                ("on_gpu", ctypes.c_int), ("start_ms", ctypes.c_double), ("done_ms", ctypes.c_double)]


HOST_ENGINE_FN = ctypes.CFUNCTYPE(ctypes.c_int, ctypes.c_void_p, ctypes.POINTER(olap_serve_request))


class olap_serve_opts(ctypes.Structure):
    _fields_ = [("policy", ctypes.c_int), ("gpu_slots", ctypes.c_int), ("cpu_workers", ctypes.c_int),
                ("mem_budget_bytes", ctypes.c_uint64), ("topk_model", ctypes.c_void_p),
                ("probe_model", ctypes.c_void_p), ("host_engine", ctypes.c_void_p), ("host_user", ctypes.c_void_p),
                ("closed_loop", ctypes.c_int), ("ctx_opts", ctypes.c_void_p)]


class olap_serve_stats(ctypes.Structure):
    _fields_ = [(nm, ctypes.c_double) for nm in ("wall_ms", "throughput_rps", "p50_ms", "p95_ms", "p99_ms",
                                                  "mean_ms", "max_ms")] + \
        [("n_gpu", ctypes.c_uint64), ("n_host", ctypes.c_uint64), ("n_failed", ctypes.c_uint64),
         ("offload_fraction", ctypes.c_double), ("peak_reserved_bytes", ctypes.c_uint64)]


class olap_topk_info(ctypes.Structure):
    _fields_ = [
        ("path", ctypes.c_int),
        ("refine_passes", ctypes.c_int),
        ("candidates", ctypes.c_uint64),
        ("phase_ns", ctypes.c_uint64 * 8),
        ("rowids_in_place", ctypes.c_int),
        ("reserved", ctypes.c_int),
    ]


class olap_tune_request(ctypes.Structure):
    _fields_ = [("topk_n", ctypes.c_uint64), ("topk_key_type", ctypes.c_int), ("reps", ctypes.c_int),
                ("topk_k", ctypes.c_uint64), ("join_build_n", ctypes.c_uint64), ("join_probe_n", ctypes.c_uint64),
                ("join_hit_rate", ctypes.c_double), ("seed", ctypes.c_uint64)]


class olap_tune_result(ctypes.Structure):
    _fields_ = [("block_threads", ctypes.c_int), ("topk_digit_bits", ctypes.c_int), ("topk_ms", ctypes.c_double),
                ("topk_default_ms", ctypes.c_double), ("load_factor", ctypes.c_double),
                ("join_partitions", ctypes.c_int), ("join_bucket_loads", ctypes.c_int),
                ("join_probe_ms", ctypes.c_double), ("join_probe_default_ms", ctypes.c_double),
                ("join_build_ms", ctypes.c_double), ("candidates", ctypes.c_int), ("pad", ctypes.c_int)]


class olap_kernel_ms(ctypes.Structure):
    _fields_ = [(nm, ctypes.c_float) for nm in
                ("topk_prepare_ms", "topk_filter_ms", "topk_select_ms", "join_probe_ms")]


_lib = None
_lock = threading.Lock()


def lib_path() -> str:
    return _build.LIB


def load(path: str | None = None):
    """Load libolap.so (built in-tree by ``build.build()``); raise if absent."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        p = path or lib_path()
        if not os.path.exists(p):
            raise ImportError(f"CUDA library not built: {p} is missing (run __graft_entry__.build())")
        lib = ctypes.CDLL(p)
        vp, u64, i32 = ctypes.c_void_p, ctypes.c_uint64, ctypes.c_int
        lib.olap_ctx_create.restype = i32
        lib.olap_ctx_create.argtypes = [ctypes.POINTER(olap_opts), ctypes.POINTER(vp)]
        lib.olap_ctx_destroy.restype = None
        lib.olap_ctx_destroy.argtypes = [vp]
        lib.olap_last_error.restype = ctypes.c_char_p
        lib.olap_last_error.argtypes = [vp]
        lib.olap_ctx_stream.restype = vp
        lib.olap_ctx_stream.argtypes = [vp]
        lib.olap_ctx_sync.restype = i32
        lib.olap_ctx_sync.argtypes = [vp]
        lib.olap_ctx_host_direct.restype = i32
        lib.olap_ctx_host_direct.argtypes = [vp]
        lib.olap_selftest_wait.restype = i32
        lib.olap_selftest_wait.argtypes = [vp, u64, ctypes.POINTER(ctypes.c_int32)]
        lib.olap_topk.restype = i32
        lib.olap_topk.argtypes = [vp, vp, i32, vp, i32, u64, u64, i32, vp, vp, i32, ctypes.POINTER(u64)]
        lib.olap_topk_pair.restype = i32
        lib.olap_topk_pair.argtypes = [vp, vp, i32, i32, vp, i32, i32, vp, i32, u64, u64, vp, vp, vp, i32,
                                       ctypes.POINTER(u64)]
        lib.olap_topk_async.restype = i32
        lib.olap_topk_async.argtypes = [vp, vp, i32, vp, u64, u64, i32, vp, vp, vp, vp]
        lib.olap_topk_rows.restype = i32
        lib.olap_topk_rows.argtypes = [vp, vp, i32, u64, ctypes.c_uint32, ctypes.c_uint32, i32, u64, i32, vp, vp,
                                       i32, ctypes.POINTER(u64)]
        lib.olap_topk_info_last.restype = i32
        lib.olap_topk_info_last.argtypes = [vp, ctypes.POINTER(olap_topk_info)]
        lib.olap_autotune.restype = i32
        lib.olap_autotune.argtypes = [vp, ctypes.POINTER(olap_tune_request), ctypes.POINTER(olap_tune_result)]
        lib.olap_ctx_time_kernels.restype = i32
        lib.olap_ctx_time_kernels.argtypes = [vp, i32]
        lib.olap_kernel_ms_last.restype = i32
        lib.olap_kernel_ms_last.argtypes = [vp, ctypes.POINTER(olap_kernel_ms)]
        lib.olap_ctx_launches.restype = i32
        lib.olap_ctx_launches.argtypes = [vp, ctypes.POINTER(u64)]
        lib.olap_join_build.restype = i32
        lib.olap_join_build.argtypes = [vp, vp, vp, i32, u64, ctypes.c_double, ctypes.POINTER(vp)]
        lib.olap_join_probe.restype = i32
        lib.olap_join_probe.argtypes = [vp, vp, vp, vp, i32, u64, vp, i32, u64, ctypes.POINTER(u64)]
        lib.olap_join_probe_async.restype = i32
        lib.olap_join_probe_async.argtypes = [vp, vp, vp, vp, u64, vp, u64, vp, vp]
        lib.olap_join_probe_partitions.restype = i32
        lib.olap_join_probe_partitions.argtypes = [vp, vp, u64, ctypes.POINTER(ctypes.c_int)]
        lib.olap_join_probe_info_last.restype = i32
        lib.olap_join_probe_info_last.argtypes = [vp, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                                                  ctypes.POINTER(u64)]
        lib.olap_join_table_info.restype = i32
        lib.olap_join_table_info.argtypes = [vp, ctypes.POINTER(u64), ctypes.POINTER(u64), ctypes.POINTER(u64),
                                             ctypes.POINTER(u64)]
        lib.olap_join_free.restype = None
        lib.olap_join_free.argtypes = [vp]
        lib.olap_gate_calibrate.restype = i32
        lib.olap_gate_calibrate.argtypes = [ctypes.POINTER(olap_gate_samples), ctypes.c_double,
                                            ctypes.POINTER(olap_gate_model)]
        lib.olap_gate_estimate.restype = i32
        lib.olap_gate_estimate.argtypes = [ctypes.POINTER(olap_gate_model), ctypes.POINTER(olap_gate_query),
                                           ctypes.POINTER(olap_gate_decision)]
        lib.olap_batch_create.restype = i32
        lib.olap_batch_create.argtypes = [vp, ctypes.POINTER(olap_batch_item), u64, ctypes.POINTER(vp)]
        lib.olap_batch_run.restype = i32
        lib.olap_batch_run.argtypes = [vp, vp]
        lib.olap_batch_run_per_query.restype = i32
        lib.olap_batch_run_per_query.argtypes = [vp, vp]
        lib.olap_batch_errors.restype = i32
        lib.olap_batch_errors.argtypes = [vp, ctypes.POINTER(ctypes.c_int)]
        lib.olap_batch_free.restype = None
        lib.olap_batch_free.argtypes = [vp]
        lib.olap_serve.restype = i32
        lib.olap_serve.argtypes = [ctypes.POINTER(olap_serve_request), u64, ctypes.POINTER(olap_serve_opts),
                                   ctypes.POINTER(olap_serve_stats)]
        lib.olap_topk_noalloc.restype = i32
        lib.olap_topk_noalloc.argtypes = [vp, i32, vp, u64, u64, i32, vp, vp, vp, vp]
        _bind_more(lib)
        _lib = lib
        return lib


def _bind_more(lib):
    """Bindings of the entry points added after Top-K (join, gate, batch)."""
    for fn in _EXTRA_BINDERS:
        fn(lib)


_EXTRA_BINDERS = []


# ---------------------------------------------------------------------------
# Buffer marshalling
# ---------------------------------------------------------------------------

def _torch():
    import torch  # noqa: WPS433 (torch is only plumbing: memory and streams)
    return torch


def mem_kind(buf) -> int:
    if isinstance(buf, np.ndarray):
        return MEM_HOST
    torch = _torch()
    if isinstance(buf, torch.Tensor):
        if buf.is_cuda:
            return MEM_DEVICE
        return MEM_HOST_PINNED if buf.is_pinned() else MEM_HOST
    raise TypeError(f"unsupported buffer type {type(buf)}")


def ptr(buf) -> int | None:
    if buf is None:
        return None
    if isinstance(buf, np.ndarray):
        if not buf.flags["C_CONTIGUOUS"]:
            raise ValueError("buffers must be C-contiguous")
        return buf.ctypes.data
    if not buf.is_contiguous():
        raise ValueError("tensors must be contiguous")
    return buf.data_ptr()


def _check_rowids(rowids, where: int, n: int) -> None:
    """Explicit row-ids must sit in the same kind of memory as the keys and
    hold one entry per key."""
    if rowids is None:
        return
    if mem_kind(rowids) != where:
        raise ValueError("row-ids must be in the same kind of memory as the keys")
    if numel(rowids) != n:
        raise ValueError(f"{numel(rowids)} row-ids for {n} keys")


def _check_count(got: int, want: int) -> None:
    if got != want:
        raise RuntimeError(f"the library returned {got} results where {want} were due")


def key_type_of(buf) -> int:
    dt = buf.dtype
    if isinstance(buf, np.ndarray):
        for kind, npdt in KEY_NUMPY.items():
            if dt == npdt:
                return kind
    else:
        torch = _torch()
        names = {KEY_I64: "int64", KEY_F32: "float32", KEY_F64: "float64", KEY_U64: "uint64",
                 KEY_I32: "int32", KEY_U32: "uint32"}
        for kind, nm in names.items():
            if getattr(torch, nm, None) is not None and dt == getattr(torch, nm):
                return kind
    raise TypeError(f"keys must be int64, float32, float64, uint64, int32 or uint32, got {dt}")


def numel(buf) -> int:
    return int(buf.shape[0]) if isinstance(buf, np.ndarray) else int(buf.numel())


# ---------------------------------------------------------------------------
# Context
# ---------------------------------------------------------------------------

class Context:
    """An ``olap_ctx`` (one device, one stream, its scratch and staging)."""

    def __init__(self, device: int = 0, stream: int | None = None, mem_budget_bytes: int = 0,
                 margin_ms: float = 0.0, load_factor: float = 0.0, staging_bytes: int = 0,
                 topk_filter: int = FILTER_AUTO, topk_tile_bytes: int = 0, topk_stages: int = 0,
                 topk_ctas_per_sm: int = 0, join_partitions: int = 0, join_bucket_loads: int = 0,
                 l2_fetch_bytes: int = 0, topk_digit_bits: int = 0, block_threads: int = 0,
                 host_access: int = 0, batch_overlap: int = 0, batch_topk_ctas_per_sm: int = 0,
                 join_prefilter: int = PREFILTER_AUTO, staging_threads: int = 0):
        self.lib = load()
        opts = olap_opts(device, stream, mem_budget_bytes, margin_ms, block_threads, load_factor, staging_bytes,
                         topk_filter, topk_tile_bytes, topk_stages, topk_ctas_per_sm, join_partitions,
                         join_bucket_loads, l2_fetch_bytes, topk_digit_bits, host_access, batch_overlap,
                         batch_topk_ctas_per_sm, join_prefilter, staging_threads)
        h = ctypes.c_void_p()
        st = self.lib.olap_ctx_create(ctypes.byref(opts), ctypes.byref(h))
        if st != OK:
            raise OlapError(st, "olap_ctx_create failed (no usable CUDA device?)")
        self.h = h

    def close(self):
        if getattr(self, "h", None):
            self.lib.olap_ctx_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    @property
    def stream(self) -> int:
        return self.lib.olap_ctx_stream(self.h)

    def last_error(self) -> str:
        return self.lib.olap_last_error(self.h).decode()

    def check(self, st: int):
        if st != OK:
            raise OlapError(st, self.last_error())

    def sync(self):
        self.check(self.lib.olap_ctx_sync(self.h))

    def _after_torch(self, *bufs, stream: int | None = None, force: bool = False):
        """Order the library's stream (`stream`, else the context's) after the
        work queued on torch's current stream, when a buffer is a CUDA tensor
        (or `force`): the library runs on its own non-blocking stream, so a
        tensor that torch is still writing would otherwise be read early, and
        one that torch is still clearing (a count, a status word) could be
        cleared after the library wrote it."""
        if not force and not any(b is not None and mem_kind(b) == MEM_DEVICE for b in bufs
                                 if not isinstance(b, np.ndarray)):
            return
        torch = _torch()
        cur = torch.cuda.current_stream()
        target = self.stream if stream is None else int(stream)
        # nothing to wait for when torch's stream has finished its work (a
        # host-side query; a wait on the GPU costs the call a few us)
        if target != cur.cuda_stream and not cur.query():
            torch.cuda.ExternalStream(target).wait_stream(cur)

    # -- Top-K ---------------------------------------------------------------
    def topk(self, keys, k: int, order: int = DESC, rowids=None, out_keys=None, out_rowids=None):
        """olap_topk: returns (out_keys, out_rowids) cut to min(k, n).

        Outputs default to numpy arrays (host); pass preallocated buffers
        (numpy, pinned or CUDA torch tensors) to choose their memory kind."""
        n = numel(keys)
        kt = key_type_of(keys)
        cnt = min(int(k), n)
        if out_keys is None:
            out_keys = np.empty(max(cnt, 1), dtype=KEY_NUMPY[kt])
            out_rowids = np.empty(max(cnt, 1), dtype=np.uint32)
        where = mem_kind(keys)
        _check_rowids(rowids, where, n)
        ow = mem_kind(out_keys)
        self._after_torch(keys, rowids, out_keys, out_rowids)
        got = ctypes.c_uint64()
        st = self.lib.olap_topk(self.h, ptr(keys), kt, ptr(rowids), where, n, int(k), int(order),
                                ptr(out_keys), ptr(out_rowids), ow, ctypes.byref(got))
        self.check(st)
        _check_count(got.value, cnt)
        return out_keys[:cnt], out_rowids[:cnt]

    def topk_pair(self, keys0, order0: int, keys1, order1: int, k: int, rowids=None, out_keys0=None,
                  out_keys1=None, out_rowids=None):
        """olap_topk_pair (ORDER BY c0, c1 LIMIT k over two 4-byte key
        columns): returns (c0 keys, c1 keys, row-ids) cut to min(k, n)."""
        n = numel(keys0)
        if numel(keys1) != n:
            raise ValueError("both key columns must hold the same number of rows")
        where = mem_kind(keys0)
        if mem_kind(keys1) != where:
            raise ValueError("both key columns must be in the same kind of memory")
        _check_rowids(rowids, where, n)
        t0, t1 = key_type_of(keys0), key_type_of(keys1)
        cnt = min(int(k), n)
        if out_keys0 is None:
            out_keys0 = np.empty(max(cnt, 1), dtype=KEY_NUMPY[t0])
            out_keys1 = np.empty(max(cnt, 1), dtype=KEY_NUMPY[t1])
            out_rowids = np.empty(max(cnt, 1), dtype=np.uint32)
        self._after_torch(keys0, keys1, rowids, out_keys0, out_keys1, out_rowids)
        got = ctypes.c_uint64()
        st = self.lib.olap_topk_pair(self.h, ptr(keys0), t0, int(order0), ptr(keys1), t1, int(order1), ptr(rowids),
                                     where, n, int(k), ptr(out_keys0), ptr(out_keys1), ptr(out_rowids),
                                     mem_kind(out_keys0), ctypes.byref(got))
        self.check(st)
        _check_count(got.value, cnt)
        return out_keys0[:cnt], out_keys1[:cnt], out_rowids[:cnt]

    def topk_rows(self, rows, row_bytes: int, key_offset: int, key_type: int, k: int, order: int = DESC,
                  out_rows=None, out_rowids=None):
        """olap_topk_rows (full-row offload): `rows` holds n rows of row_bytes
        bytes (numpy, pinned or CUDA tensor); returns (rows, row-ids) of the
        min(k, n) selected rows, whole."""
        nbytes = rows.nbytes if isinstance(rows, np.ndarray) else rows.numel() * rows.element_size()
        if row_bytes <= 0 or nbytes % row_bytes:
            raise ValueError("the row buffer must hold a whole number of rows")
        n = nbytes // row_bytes
        cnt = min(int(k), n)
        if out_rows is None:
            out_rows = np.empty(max(cnt, 1) * row_bytes, dtype=np.uint8)
            out_rowids = np.empty(max(cnt, 1), dtype=np.uint32)
        self._after_torch(rows, out_rows, out_rowids)
        got = ctypes.c_uint64()
        self.check(self.lib.olap_topk_rows(self.h, ptr(rows), mem_kind(rows), n, row_bytes, key_offset, key_type,
                                           int(k), int(order), ptr(out_rows), ptr(out_rowids), mem_kind(out_rows),
                                           ctypes.byref(got)))
        _check_count(got.value, cnt)
        return out_rows, (None if out_rowids is None else out_rowids[:cnt])

    # -- Join ----------------------------------------------------------------
    def join_build(self, keys, rowids=None, load_factor: float = 0.0) -> "JoinTable":
        """olap_join_build over int64 keys (numpy, pinned or CUDA tensor)."""
        where = mem_kind(keys)
        _check_rowids(rowids, where, numel(keys))
        self._after_torch(keys, rowids)
        h = ctypes.c_void_p()
        self.check(self.lib.olap_join_build(self.h, ptr(keys), ptr(rowids), where, numel(keys),
                                            float(load_factor), ctypes.byref(h)))
        return JoinTable(self.lib, h)

    def join_probe(self, table: "JoinTable", keys, rowids=None, out=None, capacity: int | None = None):
        """olap_join_probe.  Returns the pairs as an (M, 2) uint32 array
        [probe_rowid, build_rowid] (numpy by default, or the given buffer cut to
        M rows).  With no buffer given, retries once with the exact size when
        the first guess overflows."""
        where = mem_kind(keys)
        n = numel(keys)
        _check_rowids(rowids, where, n)
        own = out is None
        if own:
            capacity = capacity if capacity is not None else max(16, 2 * n)
            out = np.empty((capacity, 2), dtype=np.uint32)
        cap = (out.shape[0] if isinstance(out, np.ndarray) else out.numel() // 2) if capacity is None else capacity
        self._after_torch(keys, rowids, out)
        got = ctypes.c_uint64()
        st = self.lib.olap_join_probe(self.h, table.h, ptr(keys), ptr(rowids), where, n, ptr(out), mem_kind(out),
                                      cap, ctypes.byref(got))
        if st == E_OVERFLOW and own:
            out = np.empty((max(1, got.value), 2), dtype=np.uint32)
            st = self.lib.olap_join_probe(self.h, table.h, ptr(keys), ptr(rowids), where, n, ptr(out),
                                          MEM_HOST, got.value, ctypes.byref(got))
        if st == E_OVERFLOW:
            raise OlapError(st, f"{self.last_error()} (need {got.value} pairs)")
        self.check(st)
        return out[: got.value]

    def join_probe_async(self, table: "JoinTable", d_keys, d_out, capacity: int, d_count, d_rowids=None,
                         stream: int | None = None):
        self._after_torch(d_keys, stream=stream, force=True)
        self.check(self.lib.olap_join_probe_async(self.h, table.h, ptr(d_keys), ptr(d_rowids), numel(d_keys),
                                                  ptr(d_out), int(capacity), ptr(d_count), stream))

    # -- Batched executor ----------------------------------------------------
    def join_probe_partitions(self, table: "JoinTable", n: int) -> int:
        """olap_join_probe_partitions: 1 for the direct probe, else the radix
        partitions a probe of n rows against `table` uses on this context."""
        parts = ctypes.c_int()
        self.check(self.lib.olap_join_probe_partitions(self.h, table.h, int(n), ctypes.byref(parts)))
        return parts.value

    def join_probe_info(self) -> dict:
        """olap_join_probe_info_last: partitions, whether the Bloom pre-probe
        dropped rows, and the rows left to probe, of the last probe."""
        parts, pf, rows = ctypes.c_int(), ctypes.c_int(), ctypes.c_uint64()
        self.check(self.lib.olap_join_probe_info_last(self.h, ctypes.byref(parts), ctypes.byref(pf),
                                                      ctypes.byref(rows)))
        return {"parts": parts.value, "prefiltered": bool(pf.value), "rows_probed": rows.value}

    def batch(self, items) -> "Batch":
        """olap_batch_create from a list of olap_batch_item."""
        arr = (olap_batch_item * max(1, len(items)))(*items)
        h = ctypes.c_void_p()
        self.check(self.lib.olap_batch_create(self.h, arr, len(items), ctypes.byref(h)))
        return Batch(self, h)

    def topk_info(self) -> dict:
        """olap_topk_info_last as a dict (phase times in microseconds)."""
        info = olap_topk_info()
        self.check(self.lib.olap_topk_info_last(self.h, ctypes.byref(info)))
        names = ["sample", "filter", "refine", "split", "finish", "total", "finish_small", "finish_sort"]
        return {"path": info.path, "refine_passes": info.refine_passes, "candidates": info.candidates,
                "rowids_in_place": bool(info.rowids_in_place),
                "phase_us": {nm: info.phase_ns[i] / 1e3 for i, nm in enumerate(names)}}

    def autotune(self, topk_n: int = 0, topk_k: int = 100, key_type: int = KEY_I64, join_build_n: int = 0,
                 join_probe_n: int = 0, join_hit_rate: float = 0.5, reps: int = 5, seed: int = 7) -> dict:
        """olap_autotune: time candidate configurations on this shape and keep
        the fastest in this context; returns the olap_tune_result as a dict."""
        req = olap_tune_request(topk_n, key_type, reps, topk_k, join_build_n, join_probe_n, join_hit_rate, seed)
        res = olap_tune_result()
        self.check(self.lib.olap_autotune(self.h, ctypes.byref(req), ctypes.byref(res)))
        return {nm: getattr(res, nm) for nm, _ in olap_tune_result._fields_ if nm != "pad"}

    def selftest_wait(self, limit_cycles: int) -> int:
        """olap_selftest_wait: the device status a bounded wait on a word that
        nothing writes records (OLAP_E_TIMEOUT expected)."""
        st = ctypes.c_int32(-1)
        self.check(self.lib.olap_selftest_wait(self.h, int(limit_cycles), ctypes.byref(st)))
        return st.value

    @property
    def host_direct(self) -> bool:
        """Whether pageable host memory is copied by a kernel reading it directly."""
        return bool(self.lib.olap_ctx_host_direct(self.h))

    def time_kernels(self, on: bool = True):
        """olap_ctx_time_kernels: record CUDA events around each kernel."""
        self.check(self.lib.olap_ctx_time_kernels(self.h, 1 if on else 0))

    def launches(self) -> int:
        """olap_ctx_launches: kernels launched for this context so far."""
        c = ctypes.c_uint64()
        self.check(self.lib.olap_ctx_launches(self.h, ctypes.byref(c)))
        return c.value

    def kernel_ms(self) -> dict:
        """olap_kernel_ms_last as a dict (milliseconds; -1 = not timed)."""
        t = olap_kernel_ms()
        self.check(self.lib.olap_kernel_ms_last(self.h, ctypes.byref(t)))
        return {nm: getattr(t, nm) for nm, _ in olap_kernel_ms._fields_}

    def topk_async(self, d_keys, k: int, order: int, d_out_keys, d_out_rowids, d_rowids=None,
                   dev_status=None, stream: int | None = None):
        """olap_topk_async on CUDA tensors; enqueues only."""
        self._after_torch(d_keys, stream=stream, force=True)
        st = self.lib.olap_topk_async(self.h, ptr(d_keys), key_type_of(d_keys), ptr(d_rowids),
                                      numel(d_keys), int(k), int(order), ptr(d_out_keys),
                                      ptr(d_out_rowids), ptr(dev_status), stream)
        self.check(st)


class Batch:
    """A captured batch (olap_batch): run() replays its CUDA graph."""

    def __init__(self, ctx: "Context", h):
        self.ctx = ctx
        self.h = h

    def run(self, stream: int | None = None):
        self.ctx._after_torch(stream=stream, force=True)
        self.ctx.check(self.ctx.lib.olap_batch_run(self.h, stream))

    def run_per_query(self, stream: int | None = None):
        self.ctx._after_torch(stream=stream, force=True)
        self.ctx.check(self.ctx.lib.olap_batch_run_per_query(self.h, stream))

    def errors(self) -> int:
        e = ctypes.c_int()
        self.ctx.check(self.ctx.lib.olap_batch_errors(self.h, ctypes.byref(e)))
        return e.value

    def free(self):
        if getattr(self, "h", None):
            self.ctx.lib.olap_batch_free(self.h)
            self.h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def topk_item(d_keys, k: int, order: int, d_out_keys, d_out_rowids, d_count, d_rowids=None, d_status=None):
    return olap_batch_item(OP_TOPK, key_type_of(d_keys), order, ptr(d_keys), ptr(d_rowids), numel(d_keys), k,
                           ptr(d_out_keys), ptr(d_out_rowids), None, None, 0, ptr(d_count), ptr(d_status))


def probe_item(table: "JoinTable", d_keys, d_out_pairs, capacity: int, d_count, d_rowids=None, d_status=None):
    return olap_batch_item(OP_PROBE, KEY_I64, 0, ptr(d_keys), ptr(d_rowids), numel(d_keys), 0, None, None,
                           table.h.value if isinstance(table.h, ctypes.c_void_p) else table.h, ptr(d_out_pairs),
                           capacity, ptr(d_count), ptr(d_status))


class JoinTable:
    """A resident key-only hash table (olap_join_table)."""

    def __init__(self, lib, h):
        self.lib = lib
        self.h = h

    def info(self) -> dict:
        nb, nk, ns, bb = ctypes.c_uint64(), ctypes.c_uint64(), ctypes.c_uint64(), ctypes.c_uint64()
        st = self.lib.olap_join_table_info(self.h, ctypes.byref(nb), ctypes.byref(nk), ctypes.byref(ns),
                                           ctypes.byref(bb))
        if st != OK:
            raise OlapError(st, "olap_join_table_info failed")
        return {"n_build": nb.value, "n_buckets": nk.value, "n_side": ns.value, "bloom_bytes": bb.value}

    def has_bloom(self) -> bool:
        return self.info()["bloom_bytes"] > 0

    def free(self):
        if getattr(self, "h", None):
            self.lib.olap_join_free(self.h)
            self.h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def topk_noalloc(d_keys, k: int, order: int, d_out_keys, d_out_rowids, d_rowids=None, dev_status=None,
                 stream: int | None = None):
    """olap_topk_noalloc on CUDA tensors of the current device: the Top-K for
    callers that cannot let the library allocate device memory (its working
    memory is a fixed array inside the library).  Enqueues only."""
    lib = load()
    n = numel(d_keys)
    if n > NOALLOC_MAX_N or int(k) > NOALLOC_MAX_K:
        raise ValueError(f"olap_topk_noalloc handles n <= {NOALLOC_MAX_N} and k <= {NOALLOC_MAX_K}; "
                         f"got n={n}, k={k}")
    if int(k) < 0 or int(order) not in (ASC, DESC):
        raise ValueError(f"bad k={k} or order={order}")
    cnt = min(int(k), n)
    for nm, buf in (("d_keys", d_keys), ("d_out_keys", d_out_keys), ("d_out_rowids", d_out_rowids),
                    ("d_rowids", d_rowids), ("dev_status", dev_status)):
        if buf is not None and mem_kind(buf) != MEM_DEVICE:
            raise ValueError(f"{nm} must be a CUDA tensor")
    if cnt and (d_out_keys is None or d_out_rowids is None):
        raise ValueError("output buffers are required when min(k, n) > 0")
    if cnt and (numel(d_out_keys) < cnt or numel(d_out_rowids) < cnt):
        raise ValueError(f"outputs must hold min(k, n) = {cnt} entries")
    if d_rowids is not None and numel(d_rowids) != n:
        raise ValueError(f"{numel(d_rowids)} row-ids for {n} keys")
    st = lib.olap_topk_noalloc(ptr(d_keys), key_type_of(d_keys), ptr(d_rowids), n, int(k), int(order),
                               ptr(d_out_keys), ptr(d_out_rowids), ptr(dev_status), stream)
    if st != OK:
        raise OlapError(st, "olap_topk_noalloc failed")


# ---------------------------------------------------------------------------
# Risky Gate (host arithmetic in the library; no device needed)
# ---------------------------------------------------------------------------

def gate_calibrate(op: int, n, k_or_m, tx_bytes, out_rows, t_cpu_ms, t_tx_ms, t_ker_ms, t_post_ms,
                   margin_ms: float = 0.0, weighting: int = FIT_ORDINARY, topk_cpu: int = 0,
                   cpu_split_n: float = 0.0) -> olap_gate_model:
    """olap_gate_calibrate over equal-length sample sequences (times in ms);
    cpu_split_n > 0 fits the CPU cost separately below and above that size."""
    lib = load()
    cols = [np.ascontiguousarray(np.asarray(c, dtype=np.float64)) for c in
            (n, k_or_m, tx_bytes, out_rows, t_cpu_ms, t_tx_ms, t_ker_ms, t_post_ms)]
    cnt = cols[0].shape[0]
    if any(c.shape[0] != cnt for c in cols):
        raise ValueError("every sample sequence must have the same length")
    ptrs = [c.ctypes.data_as(_dp) for c in cols]
    smp = olap_gate_samples(op, weighting, cnt, *ptrs, topk_cpu, 0, float(cpu_split_n))
    m = olap_gate_model()
    st = lib.olap_gate_calibrate(ctypes.byref(smp), float(margin_ms), ctypes.byref(m))
    if st != OK:
        raise OlapError(st, "olap_gate_calibrate rejected the samples")
    return m


def gate_estimate(model: olap_gate_model, op: int, n: int, k_or_m: float, tx_bytes: float, out_rows: float,
                  bytes_per_row: float = 0.0, out_per_row: float = 0.0) -> olap_gate_decision:
    lib = load()
    q = olap_gate_query(op, int(n), float(k_or_m), float(tx_bytes), float(out_rows), float(bytes_per_row),
                        float(out_per_row))
    d = olap_gate_decision()
    st = lib.olap_gate_estimate(ctypes.byref(model), ctypes.byref(q), ctypes.byref(d))
    if st != OK:
        raise OlapError(st, "olap_gate_estimate rejected the query")
    return d


# ---------------------------------------------------------------------------
# Serving loop and the host engine of the serving harness
# ---------------------------------------------------------------------------

class HostEngine:
    """The serving harness's CPU engine (libolap_host.so): the existing
    engine the GPU augments, used for requests the gate keeps on the host."""

    def __init__(self, threads: int = 8, cpus=None):
        """`threads` workers; with `cpus` (host core numbers), the engine
        computes only on those cores, callers' threads included."""
        p = _build.HOST_LIB
        if not os.path.exists(p):
            raise ImportError(f"host engine not built: {p} is missing")
        self.lib = ctypes.CDLL(p)
        self.lib.olap_host_engine_create.restype = ctypes.c_void_p
        self.lib.olap_host_engine_create.argtypes = [ctypes.c_int]
        self.lib.olap_host_engine_create_on.restype = ctypes.c_void_p
        self.lib.olap_host_engine_create_on.argtypes = [ctypes.c_int, ctypes.POINTER(ctypes.c_int), ctypes.c_int]
        self.lib.olap_host_engine_add_table.restype = ctypes.c_int
        self.lib.olap_host_engine_add_table.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                                        ctypes.c_uint64]
        self.lib.olap_host_engine_free.argtypes = [ctypes.c_void_p]
        self.lib.olap_host_engine_extract.restype = None
        self.lib.olap_host_engine_extract.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_uint64, ctypes.c_uint32,
                                                      ctypes.c_uint32, ctypes.c_uint32, ctypes.c_void_p]
        self.lib.olap_host_engine_parallel_from.restype = ctypes.c_uint64
        self.lib.olap_host_engine_parallel_from.argtypes = [ctypes.c_void_p, ctypes.c_int]
        if cpus:
            arr = (ctypes.c_int * len(cpus))(*[int(c) for c in cpus])
            self.h = self.lib.olap_host_engine_create_on(threads, arr, len(cpus))
        else:
            self.h = self.lib.olap_host_engine_create(threads)
        self.cpus = list(cpus) if cpus else None
        self._keep = []

    def parallel_from(self, op: int) -> int:
        """Smallest request size the engine splits over threads (0: never):
        where its cost changes regime."""
        return int(self.lib.olap_host_engine_parallel_from(self.h, int(op)))

    def add_table(self, keys: np.ndarray, rowids: np.ndarray | None = None) -> int:
        keys = np.ascontiguousarray(keys, dtype=np.int64)
        return self.lib.olap_host_engine_add_table(self.h, keys.ctypes.data, ptr(rowids), keys.shape[0])

    @property
    def fn(self) -> int:
        return ctypes.cast(self.lib.olap_host_engine_run, ctypes.c_void_p).value

    def run(self, req: olap_serve_request) -> int:
        f = ctypes.CFUNCTYPE(ctypes.c_int, ctypes.c_void_p, ctypes.POINTER(olap_serve_request))(self.fn)
        return f(self.h, ctypes.byref(req))

    def extract(self, rows: np.ndarray, row_bytes: int, key_offset: int, dtype) -> np.ndarray:
        """The key column of a row table (one field per row), cut out on the
        engine's threads."""
        n = rows.nbytes // row_bytes
        out = np.empty(n, dtype=dtype)
        self.lib.olap_host_engine_extract(self.h, rows.ctypes.data, n, row_bytes, key_offset, out.itemsize,
                                          out.ctypes.data)
        return out

    def close(self):
        if getattr(self, "h", None):
            self.lib.olap_host_engine_free(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def serve(requests, policy: int, topk_model=None, probe_model=None, host: HostEngine | None = None,
          gpu_slots: int = 4, cpu_workers: int = 8, mem_budget_bytes: int = 0, closed_loop: bool = False,
          device: int = 0, host_access: int = HOST_AUTO) -> olap_serve_stats:
    """olap_serve over a ctypes array (or list) of olap_serve_request; the
    slot contexts are created with the given host_access."""
    lib = load()
    arr = requests if isinstance(requests, ctypes.Array) else (olap_serve_request * len(requests))(*requests)
    co = olap_opts(device=device, host_access=host_access)
    o = olap_serve_opts(policy, gpu_slots, cpu_workers, mem_budget_bytes,
                        ctypes.addressof(topk_model) if topk_model is not None else None,
                        ctypes.addressof(probe_model) if probe_model is not None else None,
                        host.fn if host else None, host.h if host else None, 1 if closed_loop else 0,
                        ctypes.addressof(co))
    st = olap_serve_stats()
    rc = lib.olap_serve(arr, len(arr), ctypes.byref(o), ctypes.byref(st))
    if rc != OK:
        raise OlapError(rc, "olap_serve failed")
    return st
