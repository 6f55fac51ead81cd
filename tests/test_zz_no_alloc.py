"""The allocation-free reduction entry point (HDArrayReduceBufferNoAlloc) against HDArrayReduce.

HDArrayReduceBufferNoAlloc serves callers that cannot call cudaMalloc -- code whose device memory
belongs to another allocator, and latency-critical paths that cannot take cudaMalloc's implicit
synchronisation.  Its scratch is a fixed static device array, so the test checks that two calls in
a row (sharing that scratch) both match the allocating entry point, and that it refuses a size
beyond its maximum.  This file is collected last on purpose.
"""
import ctypes

import numpy as np
import pytest

import synthetic

pytestmark = pytest.mark.gpu

H = pytest.importorskip("paper_1809_05657_gb300.hdarray")


@pytest.fixture
def gpu_lib():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from __graft_entry__ import build_library
    build_library()
    torch.cuda.init()
    yield torch
    H.HDArrayExit()


def _noalloc():
    f = H.lib().HDArrayReduceBufferNoAlloc
    f.restype = ctypes.c_int
    f.argtypes = [ctypes.c_void_p, ctypes.c_char_p, ctypes.c_int, ctypes.POINTER(ctypes.c_int64),
                  ctypes.POINTER(ctypes.c_int64), ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p]
    return f


@pytest.mark.parametrize("dtype", ["double", "float", "bf16"])
def test_noalloc_reduce_matches_reduce_twice(gpu_lib, dtype):
    torch = gpu_lib
    dims = (301, 517)
    u = synthetic.uniform(dims[0] * dims[1], stream=77).reshape(dims)
    x = synthetic.to_storage(1.0 + (u - 0.5) * 0.02, dtype)
    H.HDArrayInit(ndev=1)
    X = H.HDArrayCreate("X", dtype, None, *dims)
    part = H.HDArrayPartition(H.ROW, dims, (0, 0), dims, 1)
    H.HDArrayWrite(X, x, part)
    ptr, lo, hi, st = H.HDArrayGetDeviceBuffer(X, 0)
    esize = {"double": 8, "float": 4, "bf16": 2}[dtype]
    first = ptr + ((0 - lo[0]) * st[0] + (0 - lo[1]) * st[1]) * esize  # element (0, 0)
    extent = (ctypes.c_int64 * 2)(*dims)
    strides = (ctypes.c_int64 * 2)(st[0], st[1])
    out = torch.zeros(1, dtype=torch.float64, device="cuda")  # the caller owns the output
    f = _noalloc()
    for op in (H.SUM, H.MAX, H.MIN, H.PROD):
        want = H.HDArrayReduce(X, op, part)
        for _ in range(2):  # two calls in a row share the static scratch
            out.fill_(-12345.0)
            torch.cuda.synchronize()
            rc = f(first, dtype.encode(), 2, extent, strides, op, out.data_ptr(), None)
            assert rc == 0
            torch.cuda.synchronize()
            got = float(out.item())
            if op in (H.MAX, H.MIN):
                assert got == want
            else:
                assert abs(got - want) <= 1e-12 * abs(want)


def test_noalloc_rejects_oversize(gpu_lib):
    torch = gpu_lib
    buf = torch.zeros(16, dtype=torch.float32, device="cuda")
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    extent = (ctypes.c_int64 * 2)(1 << 16, (1 << 15) + 1)  # 2^31 + 2^16 elements: beyond the limit
    strides = (ctypes.c_int64 * 2)((1 << 15) + 1, 1)
    rc = _noalloc()(buf.data_ptr(), b"float", 2, extent, strides, H.SUM, out.data_ptr(), None)
    assert rc == -4  # HDARRAY_ERR_RANGE, nothing launched
