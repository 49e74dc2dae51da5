"""The C-ABI library builds, loads and exports every symbol include/olap.h
declares (no compute calls: this runs without a GPU)."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_2601_19911_gb300 import build, olap

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "olap.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[A-Za-z_][\w\s\*]*?\b(olap_\w+)\s*\(", src, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    build.build()
    return olap.load()


def test_header_declares_the_binding_exports():
    assert sorted(olap.EXPORTS) == declared_functions()


def test_every_declared_symbol_is_exported(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name
        assert ctypes.cast(getattr(lib, name), ctypes.c_void_p).value


def test_no_cpu_fallback_without_gpu(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(olap.OlapError) as ei:
        olap.Context(0)
    assert ei.value.status == olap.E_CUDA


@pytest.mark.parametrize("field,value", [("join_partitions", 3), ("join_partitions", 512), ("join_partitions", -1),
                                         ("load_factor", 0.95), ("topk_filter", 7), ("join_bucket_loads", 3),
                                         ("l2_fetch_bytes", 48), ("topk_digit_bits", 7), ("topk_digit_bits", 13),
                                         ("block_threads", 384), ("host_access", 2), ("batch_overlap", 2),
                                         ("batch_topk_ctas_per_sm", 3), ("join_prefilter", 3),
                                         ("join_prefilter", -1), ("staging_threads", -1), ("staging_threads", 65)])
def test_bad_options_are_rejected_before_any_device_call(lib, field, value):
    opts = olap.olap_opts()
    setattr(opts, field, value)
    h = ctypes.c_void_p()
    assert lib.olap_ctx_create(ctypes.byref(opts), ctypes.byref(h)) == olap.E_INVALID
    assert not h.value


def test_null_context_is_rejected(lib):
    got = ctypes.c_uint64()
    assert lib.olap_topk(None, None, 0, None, 0, 0, 0, 0, None, None, 0, ctypes.byref(got)) == olap.E_INVALID
    assert lib.olap_ctx_sync(None) == olap.E_INVALID
    assert lib.olap_last_error(None) == b"no context"


def test_struct_layouts_match_the_header(tmp_path):
    """Every ctypes mirror of an include/olap.h struct has the C layout
    (size and field offsets, from a C program compiled against the header)."""
    import subprocess
    structs = {
        "olap_opts": olap.olap_opts, "olap_topk_info": olap.olap_topk_info, "olap_kernel_ms": olap.olap_kernel_ms,
        "olap_tune_request": olap.olap_tune_request, "olap_tune_result": olap.olap_tune_result,
        "olap_gate_samples": olap.olap_gate_samples, "olap_gate_model": olap.olap_gate_model,
        "olap_gate_query": olap.olap_gate_query, "olap_gate_decision": olap.olap_gate_decision,
        "olap_batch_item": olap.olap_batch_item, "olap_serve_request": olap.olap_serve_request,
        "olap_serve_opts": olap.olap_serve_opts, "olap_serve_stats": olap.olap_serve_stats,
    }
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "olap.h"', 'int main(void) {']
    for name, cls in structs.items():
        lines.append(f'printf("{name} %zu\\n", sizeof({name}));')
        for f in cls._fields_:
            lines.append(f'printf("{name}.{f[0]} %zu\\n", offsetof({name}, {f[0]}));')
    lines.append("return 0; }")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)])
    got = dict(l.split() for l in subprocess.check_output([str(exe)], text=True).splitlines())
    for name, cls in structs.items():
        assert int(got[name]) == ctypes.sizeof(cls), name
        for f in cls._fields_:
            assert int(got[f"{name}.{f[0]}"]) == getattr(cls, f[0]).offset, (name, f[0])


def test_binding_rejects_bad_buffers_without_asserts():
    """Argument checks of the binding raise real exceptions (they survive
    python -O), before any call crosses the ABI."""
    a = np.arange(20, dtype=np.int64)
    with pytest.raises(ValueError):
        olap.ptr(a[::2])                                   # not contiguous
    olap._check_rowids(None, olap.MEM_HOST, 5)
    olap._check_rowids(np.arange(5, dtype=np.uint32), olap.MEM_HOST, 5)
    with pytest.raises(ValueError):
        olap._check_rowids(np.arange(4, dtype=np.uint32), olap.MEM_HOST, 5)
    with pytest.raises(ValueError):
        olap._check_rowids(np.arange(5, dtype=np.uint32), olap.MEM_DEVICE, 5)
    with pytest.raises(RuntimeError):
        olap._check_count(3, 4)
    with pytest.raises(ValueError):
        olap.gate_calibrate(olap.OP_TOPK, [1e3, 1e4], [10, 10], [8e3, 8e4], [10, 10], [1.0, 2.0],
                            [0.1, 0.2], [0.1, 0.1], [0.01])


def test_noalloc_refuses_bad_arguments_before_any_device_call():
    """olap_topk_noalloc checks every argument before it touches the device,
    so the refusals hold without a GPU; the addresses below are never read."""
    lib = olap.load()
    fake, odd = 0x10000, 0x10004                     # 16- and 4-byte aligned placeholders
    call = lambda keys, kt, n, k, order, ok=fake, orow=fake: lib.olap_topk_noalloc(
        keys, kt, None, n, k, order, ok, orow, None, None)
    assert call(fake, 9, 100, 10, olap.DESC) == olap.E_INVALID                   # no such key type
    assert call(fake, olap.KEY_I64, 100, 10, 7) == olap.E_INVALID               # no such order
    assert call(fake, olap.KEY_I64, olap.NOALLOC_MAX_N + 1, 10, olap.DESC) == olap.E_INVALID
    assert call(fake, olap.KEY_I64, 100, olap.NOALLOC_MAX_K + 1, olap.DESC) == olap.E_INVALID
    assert call(None, olap.KEY_I64, 100, 10, olap.DESC) == olap.E_INVALID       # keys missing
    assert call(fake, olap.KEY_I64, 100, 10, olap.DESC, ok=None) == olap.E_INVALID
    assert call(odd, olap.KEY_I64, 100, 10, olap.DESC) == olap.E_INVALID        # int64 keys 4-byte aligned
    assert call(odd + 1, olap.KEY_F32, 100, 10, olap.DESC) == olap.E_INVALID    # float32 keys misaligned
    # nothing to select and no status word: done without the device
    assert call(fake, olap.KEY_I64, 0, 10, olap.DESC) == olap.OK
    assert call(fake, olap.KEY_I64, 100, 0, olap.DESC, ok=None, orow=None) == olap.OK
