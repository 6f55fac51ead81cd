"""The allocation-free reduction entry point (HDArrayReduceBufferNoAlloc) against HDArrayReduce and
the oracle's reduction.

HDArrayReduceBufferNoAlloc serves callers that cannot call cudaMalloc -- code whose device memory
belongs to another allocator, and latency-critical paths that cannot take cudaMalloc's implicit
synchronisation.  Its scratch is a fixed static device array, so the tests check that two calls in
a row (sharing that scratch) both match the allocating entry point and the oracle, on 1-D, 2-D and
3-D boxes and an empty one, and that it refuses a size beyond its maximum.  This file is collected
last on purpose.
"""
import ctypes

import numpy as np
import pytest

import oracle
import synthetic

pytestmark = pytest.mark.gpu

H = pytest.importorskip("paper_1809_05657_gb300.hdarray")

ESIZE = {"double": 8, "float": 4, "bf16": 2}
IDENT = {0: 0.0, 1: 1.0, 2: -np.inf, 3: np.inf}


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


def _oracle_reduce(x, dtype, dims, op):
    o = oracle.Oracle(1)
    X = o.create("X", dtype, dims)
    part = o.partition(oracle.ROW, dims, (0,) * len(dims), dims, 1)
    o.write(X, x, part)
    val, _ = o.reduce(X, op, part)
    return val


def _close(got, want, op):
    if op in (H.MAX, H.MIN):
        return got == want
    return abs(got - want) <= 1e-12 * abs(want)


@pytest.mark.parametrize("dtype,dims", [("double", (301, 517)), ("float", (301, 517)), ("bf16", (301, 517)),
                                        ("float", (200_003,)), ("double", (37, 41, 53)),
                                        ("bf16", (3, 5, 20_000))])
def test_noalloc_reduce_matches_reduce_twice(gpu_lib, dtype, dims):
    torch = gpu_lib
    n = int(np.prod(dims))
    u = synthetic.uniform(n, stream=77).reshape(dims)
    x = synthetic.to_storage(1.0 + (u - 0.5) * 0.02, dtype)
    H.HDArrayInit(ndev=1)
    X = H.HDArrayCreate("X", dtype, None, *dims)
    part = H.HDArrayPartition(H.ROW, dims, (0,) * len(dims), dims, 1)
    H.HDArrayWrite(X, x, part)
    ptr, lo, hi, st = H.HDArrayGetDeviceBuffer(X, 0)
    d = len(dims)
    first = ptr + sum((0 - lo[k]) * st[k] for k in range(d)) * ESIZE[dtype]  # element (0, ..., 0)
    extent = (ctypes.c_int64 * d)(*dims)
    strides = (ctypes.c_int64 * d)(*st[:d])
    out = torch.zeros(1, dtype=torch.float64, device="cuda")  # the caller owns the output
    f = _noalloc()
    for op in (H.SUM, H.MAX, H.MIN, H.PROD):
        want = H.HDArrayReduce(X, op, part)
        ref = _oracle_reduce(x, dtype, dims, op)
        assert _close(want, ref, op)
        for _ in range(2):  # two calls in a row share the static scratch
            out.fill_(-12345.0)
            torch.cuda.synchronize()
            rc = f(first, dtype.encode(), d, extent, strides, op, out.data_ptr(), None)
            assert rc == 0
            torch.cuda.synchronize()
            got = float(out.item())
            assert _close(got, want, op), (op, got, want)
            assert _close(got, ref, op), (op, got, ref)


def test_noalloc_empty_box_gives_identity(gpu_lib):
    torch = gpu_lib
    buf = torch.ones(64, dtype=torch.float32, device="cuda")
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    f = _noalloc()
    for dims in ((0, 5), (4, 0), (0,)):
        d = len(dims)
        extent = (ctypes.c_int64 * d)(*dims)
        strides = (ctypes.c_int64 * d)(*([5] * (d - 1) + [1]))
        for op in (H.SUM, H.PROD, H.MAX, H.MIN):
            for _ in range(2):
                out.fill_(-12345.0)
                rc = f(buf.data_ptr(), b"float", d, extent, strides, op, out.data_ptr(), None)
                assert rc == 0
                torch.cuda.synchronize()
                assert float(out.item()) == IDENT[op]


def test_noalloc_rejects_oversize(gpu_lib):
    torch = gpu_lib
    # 2^16 rows of 2^15 + 1 elements = 2^31 + 2^16 elements, beyond the limit.  The outer stride is
    # 0, so every row is the same 2^15 + 1 floats of `buf`: even if the size check failed to refuse
    # the call, every access would stay inside the buffer.
    buf = torch.zeros((1 << 15) + 1, dtype=torch.float32, device="cuda")
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    extent = (ctypes.c_int64 * 2)(1 << 16, (1 << 15) + 1)
    strides = (ctypes.c_int64 * 2)(0, 1)
    rc = _noalloc()(buf.data_ptr(), b"float", 2, extent, strides, H.SUM, out.data_ptr(), None)
    assert rc == -4  # HDARRAY_ERR_RANGE, nothing launched
