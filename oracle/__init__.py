"""CPU oracle for the key-only OLAP primitives (Top-K, join, Risky Gate).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  The library under
``paper_2601_19911_gb300`` never imports it and shares no code with it.

``oracle.cpp`` (plain C++, compiled here into ``_build/liboracle.so`` with g++)
holds the Top-K (one key column or two) and join definitions; ``gate.py`` holds the gate's fits and
decision in numpy fp64.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.cpp")
_OUT = os.path.join(_HERE, "_build", "liboracle.so")
_lock = threading.Lock()
_lib = None

KEY_I64, KEY_F32, KEY_F64, KEY_U64, KEY_I32, KEY_U32 = 0, 1, 2, 3, 4, 5
_KEY_OF = {np.dtype(np.int64): KEY_I64, np.dtype(np.float32): KEY_F32, np.dtype(np.float64): KEY_F64,
           np.dtype(np.uint64): KEY_U64, np.dtype(np.int32): KEY_I32, np.dtype(np.uint32): KEY_U32}
ASC, DESC = 0, 1


def build(force: bool = False) -> str:
    """Compile oracle.cpp with the host C++ compiler (no CUDA involved)."""
    os.makedirs(os.path.dirname(_OUT), exist_ok=True)
    if force or not os.path.exists(_OUT) or os.path.getmtime(_OUT) < os.path.getmtime(_SRC):
        tmp = _OUT + f".{os.getpid()}.tmp"
        subprocess.check_call(["g++", "-O2", "-std=c++17", "-shared", "-fPIC", "-o", tmp, _SRC])
        os.replace(tmp, _OUT)
    return _OUT


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            u64, vp, i32 = ctypes.c_uint64, ctypes.c_void_p, ctypes.c_int
            lib.oracle_topk.restype = u64
            lib.oracle_topk.argtypes = [i32, vp, vp, u64, u64, i32, vp, vp]
            lib.oracle_topk_pair.restype = u64
            lib.oracle_topk_pair.argtypes = [i32, vp, i32, i32, vp, i32, vp, u64, u64, vp, vp, vp]
            for name in ("oracle_join", "oracle_join_nested"):
                fn = getattr(lib, name)
                fn.restype = u64
                fn.argtypes = [vp, vp, u64, vp, vp, u64, ctypes.POINTER(ctypes.POINTER(ctypes.c_uint64))]
            lib.oracle_free.restype = None
            lib.oracle_free.argtypes = [vp]
            lib.oracle_f32_total_below.restype = i32
            lib.oracle_f32_total_below.argtypes = [ctypes.c_uint32, ctypes.c_uint32]
            lib.oracle_f64_total_below.restype = i32
            lib.oracle_f64_total_below.argtypes = [ctypes.c_uint64, ctypes.c_uint64]
            _lib = lib
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data


def _key_type(keys: np.ndarray) -> int:
    try:
        return _KEY_OF[keys.dtype]
    except KeyError:
        raise TypeError(f"oracle keys must be int64, float32, float64, uint64, int32 or uint32, "
                        f"got {keys.dtype}") from None


def topk(keys: np.ndarray, k: int, order: int = DESC, rowids: np.ndarray | None = None):
    """First min(k, n) (key, row-id) of the (key order, row-id ascending) sort."""
    lib = _load()
    keys = np.ascontiguousarray(keys)
    n = keys.shape[0]
    if rowids is not None:
        rowids = np.ascontiguousarray(rowids, dtype=np.uint32)
        assert rowids.shape[0] == n
    cnt = min(int(k), n)
    ok = np.empty(max(cnt, 1), dtype=keys.dtype)
    orow = np.empty(max(cnt, 1), dtype=np.uint32)
    got = lib.oracle_topk(_key_type(keys), _ptr(keys), _ptr(rowids), n, int(k), int(order),
                          _ptr(ok), _ptr(orow))
    assert got == cnt
    return ok[:cnt], orow[:cnt]


def topk_pair(keys0: np.ndarray, order0: int, keys1: np.ndarray, order1: int, k: int,
              rowids: np.ndarray | None = None):
    """First min(k, n) rows of the (c0 in order0, c1 in order1, row-id
    ascending) sort: (c0 keys, c1 keys, row-ids)."""
    lib = _load()
    keys0 = np.ascontiguousarray(keys0)
    keys1 = np.ascontiguousarray(keys1)
    n = keys0.shape[0]
    assert keys1.shape[0] == n
    if rowids is not None:
        rowids = np.ascontiguousarray(rowids, dtype=np.uint32)
        assert rowids.shape[0] == n
    cnt = min(int(k), n)
    o0 = np.empty(max(cnt, 1), dtype=keys0.dtype)
    o1 = np.empty(max(cnt, 1), dtype=keys1.dtype)
    orow = np.empty(max(cnt, 1), dtype=np.uint32)
    got = lib.oracle_topk_pair(_key_type(keys0), _ptr(keys0), int(order0), _key_type(keys1), _ptr(keys1),
                               int(order1), _ptr(rowids), n, int(k), _ptr(o0), _ptr(o1), _ptr(orow))
    assert got == cnt
    return o0[:cnt], o1[:cnt], orow[:cnt]


def _join_call(fn, bkeys, brow, pkeys, prow):
    lib = _load()
    bkeys = np.ascontiguousarray(bkeys, dtype=np.int64)
    pkeys = np.ascontiguousarray(pkeys, dtype=np.int64)
    brow = None if brow is None else np.ascontiguousarray(brow, dtype=np.uint32)
    prow = None if prow is None else np.ascontiguousarray(prow, dtype=np.uint32)
    out = ctypes.POINTER(ctypes.c_uint64)()
    cnt = getattr(lib, fn)(_ptr(bkeys), _ptr(brow), bkeys.shape[0], _ptr(pkeys), _ptr(prow),
                           pkeys.shape[0], ctypes.byref(out))
    try:
        res = np.ctypeslib.as_array(out, shape=(max(cnt, 1),))[:cnt].copy()
    finally:
        lib.oracle_free(ctypes.cast(out, ctypes.c_void_p))
    return res


def join(bkeys, pkeys, brow=None, prow=None) -> np.ndarray:
    """Sorted packed pairs (probe_rowid << 32 | build_rowid), uint64."""
    return _join_call("oracle_join", bkeys, brow, pkeys, prow)


def join_nested(bkeys, pkeys, brow=None, prow=None) -> np.ndarray:
    return _join_call("oracle_join_nested", bkeys, brow, pkeys, prow)


def f32_total_below(x_bits: int, y_bits: int) -> bool:
    return bool(_load().oracle_f32_total_below(int(x_bits) & 0xFFFFFFFF, int(y_bits) & 0xFFFFFFFF))


def f64_total_below(x_bits: int, y_bits: int) -> bool:
    return bool(_load().oracle_f64_total_below(int(x_bits) & 0xFFFFFFFFFFFFFFFF, int(y_bits) & 0xFFFFFFFFFFFFFFFF))
