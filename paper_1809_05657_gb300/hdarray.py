"""Python binding of libhdarray.so: the C ABI of include/hdarray.h under the same names.

Argument marshalling only: every step of the hot path (section bookkeeping, exchange, kernels,
reductions) runs inside the library.  Arrays are passed as numpy arrays (host memory) or torch
tensors (host or CUDA memory); the library reads or writes them through their data pointers.

A call that fails raises HDArrayError with the library's error code.  Loading fails loudly when
the library has not been built (there is no fallback).
"""
import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIBPATH = os.path.join(HERE, "libhdarray.so")

HDARRAY_ROW, HDARRAY_COL, HDARRAY_BLOCK = 0, 1, 2
ROW, COL, BLOCK = HDARRAY_ROW, HDARRAY_COL, HDARRAY_BLOCK
HDARRAY_SUM, HDARRAY_PROD, HDARRAY_MAX, HDARRAY_MIN = 0, 1, 2, 3
SUM, PROD, MAX, MIN = HDARRAY_SUM, HDARRAY_PROD, HDARRAY_MAX, HDARRAY_MIN
HDARRAY_ALL = -(2 ** 31)
HDARRAY_MODE_FUSED, HDARRAY_MODE_PLAIN = 0, 1
HDARRAY_GEMM_BF16X3, HDARRAY_GEMM_BF16X6 = 2, 3
HDARRAY_INIT_HOST_ONLY = 1

ERRORS = {0: "ok", -1: "INVAL", -2: "NOMEM", -3: "RACE", -4: "RANGE", -5: "TIMEOUT", -6: "CUDA",
          -7: "STATE", -8: "UNSUPPORTED"}


class HDArrayError(RuntimeError):
    def __init__(self, code, call):
        self.code = code
        super().__init__("%s failed: %s (%d)" % (call, ERRORS.get(code, "?"), code))


_lib = None
_P = ctypes.c_void_p
_I64P = ctypes.POINTER(ctypes.c_int64)

# name -> (restype, argtypes); the variadic paper prototypes are exported too but the binding
# calls the fixed-argument forms.
SIGNATURES = {
    "HDArrayInit": (ctypes.c_int, [ctypes.c_int, _P, ctypes.c_char_p, ctypes.c_char_p]),
    "HDArrayInitEx": (ctypes.c_int, [ctypes.c_int, ctypes.c_uint]),
    "HDArrayExit": (None, []),
    "HDArrayShowDeviceInfo": (None, [ctypes.c_int]),
    "HDArrayCreatev": (_P, [ctypes.c_char_p, ctypes.c_char_p, _P, ctypes.c_int, _I64P]),
    "HDArrayFree": (ctypes.c_int, [_P]),
    "HDArrayPartitionv": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int, _I64P, _I64P, _I64P]),
    "HDArrayPartitionManual": (ctypes.c_int, [ctypes.c_int, _I64P, ctypes.c_int, _I64P, _I64P]),
    "HDArrayApplyKernelv": (ctypes.c_int, [ctypes.c_char_p, ctypes.c_int, ctypes.c_int,
                                           ctypes.POINTER(_P), ctypes.c_int,
                                           ctypes.POINTER(ctypes.c_double)]),
    "HDArrayReadv": (ctypes.c_int, [_P, _P, ctypes.c_int]),
    "HDArrayWritev": (ctypes.c_int, [_P, _P, ctypes.c_int]),
    "HDArrayReducev": (ctypes.c_int, [_P, _P, ctypes.c_int, ctypes.c_int]),
    "HDArrayReduceD": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_double), ctypes.c_int, ctypes.c_int]),
    "HDArraySetAbsoluteUsev": (ctypes.c_int, [ctypes.c_char_p, ctypes.c_int, _P, ctypes.c_int,
                                              ctypes.c_int, _I64P, _I64P]),
    "HDArraySetAbsoluteDefv": (ctypes.c_int, [ctypes.c_char_p, ctypes.c_int, _P, ctypes.c_int,
                                              ctypes.c_int, _I64P, _I64P]),
    "HDArraySetTrapezoidUsev": (ctypes.c_int, [ctypes.c_char_p, ctypes.c_int, _P, ctypes.c_int, _I64P]),
    "HDArraySetTrapezoidDefv": (ctypes.c_int, [ctypes.c_char_p, ctypes.c_int, _P, ctypes.c_int, _I64P]),
    "HDArraySetOffsetUse": (ctypes.c_int, [ctypes.c_char_p, ctypes.c_int, ctypes.c_int,
                                           ctypes.POINTER(ctypes.c_int32)]),
    "HDArraySetOffsetDef": (ctypes.c_int, [ctypes.c_char_p, ctypes.c_int, ctypes.c_int,
                                           ctypes.POINTER(ctypes.c_int32)]),
    "HDArrayNumDevices": (ctypes.c_int, []),
    "HDArraySetStream": (ctypes.c_int, [_P]),
    "HDArraySetMode": (ctypes.c_int, [ctypes.c_int]),
    "HDArraySetGemmSplit": (ctypes.c_int, [ctypes.c_int]),
    "HDArraySetAutotune": (ctypes.c_int, [ctypes.c_int]),
    "HDArrayBatchBegin": (ctypes.c_int, []),
    "HDArrayBatchEnd": (ctypes.c_int, []),
    "HDArrayGraphBegin": (ctypes.c_int, []),
    "HDArrayGraphEnd": (ctypes.c_int, [ctypes.POINTER(ctypes.c_int)]),
    "HDArrayGraphLaunch": (ctypes.c_int, [ctypes.c_int, ctypes.c_int]),
    "HDArrayGraphDestroy": (ctypes.c_int, [ctypes.c_int]),
    "HDArraySync": (ctypes.c_int, []),
    "HDArrayGetLastError": (ctypes.c_int, []),
    "HDArrayErrorString": (ctypes.c_char_p, [ctypes.c_int]),
    "HDArrayGetPlan": (ctypes.c_int64, [_P, _I64P, ctypes.c_int64]),
    "HDArrayGetGDEF": (ctypes.c_int64, [_P, ctypes.c_int, ctypes.c_int, _I64P, ctypes.c_int64]),
    "HDArrayGetDeviceBuffer": (ctypes.c_int, [_P, ctypes.c_int, ctypes.POINTER(_P), _I64P, _I64P, _I64P]),
    "HDArrayGetCounters": (ctypes.c_int, [_I64P, ctypes.c_int]),
    "HDArrayReadDeviceBuffer": (ctypes.c_int, [_P, ctypes.c_int, _I64P, _I64P, _P]),
    "HDArrayReduceBufferNoAlloc": (ctypes.c_int, [_P, ctypes.c_char_p, ctypes.c_int, _I64P, _I64P,
                                                  ctypes.c_int, _P, _P]),
    "HDArrayRegisterKernel": (ctypes.c_int, [ctypes.c_char_p, ctypes.c_int, ctypes.c_int, ctypes.c_int, _P, _P]),
    "HDArraySetAllocator": (ctypes.c_int, [_P, _P, _P]),
    "HDArraySetRankMap": (ctypes.c_int, [ctypes.c_int, ctypes.POINTER(ctypes.c_int32), ctypes.c_int]),
    "HDArraySetTransport": (ctypes.c_int, [_P, _P]),
    "HDArrayGetRankPlan": (ctypes.c_int64, [_P, _I64P, ctypes.c_int64]),
    "HDArrayStagingBytes": (ctypes.c_int64, [_P, ctypes.c_int64, _I64P]),
    "HDArrayPackBoxes": (ctypes.c_int, [_P, ctypes.c_int64, _I64P, _P, ctypes.c_int64]),
    "HDArrayUnpackBoxes": (ctypes.c_int, [_P, ctypes.c_int64, _I64P, _P, ctypes.c_int64]),
}

HDARRAY_RANK_RECORD = 10

HDARRAY_MAX_KERNEL_ARRAYS = 8


class HDArrayWork(ctypes.Structure):
    """HDArrayWork_t: one logical device's share of a call of a user kernel."""
    _fields_ = [("dev", ctypes.c_int),
                ("lo", ctypes.c_int64 * 3), ("hi", ctypes.c_int64 * 3),
                ("buf", ctypes.c_void_p * HDARRAY_MAX_KERNEL_ARRAYS),
                ("buf_lo", (ctypes.c_int64 * 3) * HDARRAY_MAX_KERNEL_ARRAYS),
                ("buf_stride", (ctypes.c_int64 * 3) * HDARRAY_MAX_KERNEL_ARRAYS)]


LAUNCHER = ctypes.CFUNCTYPE(ctypes.c_int, ctypes.POINTER(HDArrayWork), ctypes.c_int,
                            ctypes.POINTER(ctypes.c_double), ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p)
TRANSPORT = ctypes.CFUNCTYPE(ctypes.c_int, ctypes.c_void_p, ctypes.c_int64, ctypes.POINTER(ctypes.c_int64),
                             ctypes.c_void_p, ctypes.c_void_p)
ALLOC = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)
FREE = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p)
_keep = {}  # C callbacks must outlive their registration


def lib():
    """The loaded library.  Raises if it has not been built: there is no fallback path."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIBPATH):
            raise ImportError("libhdarray.so not built: run paper_1809_05657_gb300/build.py "
                              "(or __graft_entry__.build())")
        L = ctypes.CDLL(LIBPATH)
        for name, (res, args) in SIGNATURES.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _chk(rc, call):
    if rc is None or rc < 0:
        raise HDArrayError(rc if rc is not None else -1, call)
    return rc


def _i64(v):
    a = np.ascontiguousarray(np.asarray(v, dtype=np.int64).ravel())
    return a, a.ctypes.data_as(_I64P)


def _ptr(x):
    """Data pointer of a numpy array, a torch tensor, an int address or None."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if isinstance(x, np.ndarray):
        if not x.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be C-contiguous")
        return x.ctypes.data
    if hasattr(x, "data_ptr"):
        if not x.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return x.data_ptr()
    raise TypeError("unsupported buffer type %r" % type(x))


class HDArray:
    """Handle returned by HDArrayCreate."""

    def __init__(self, handle, sym, dtype, dims):
        self.handle = handle
        self.sym = sym
        self.dtype = dtype
        self.dims = tuple(dims)

    @property
    def _as_parameter_(self):
        return ctypes.c_void_p(self.handle)


# -------------------------------------------------------------------------------------------
# The paper's calls (Table 2) and the extensions, same names as the C ABI
# -------------------------------------------------------------------------------------------

def HDArrayInit(argv=None, kpath=None, dpath=None, ndev=None, host_only=False):
    if ndev is not None or host_only:
        return _chk(lib().HDArrayInitEx(ndev or 1, HDARRAY_INIT_HOST_ONLY if host_only else 0),
                    "HDArrayInitEx")
    return _chk(lib().HDArrayInit(0, None, kpath.encode() if kpath else None,
                                  dpath.encode() if dpath else None), "HDArrayInit")


def HDArrayExit():
    lib().HDArrayExit()
    _arrays.clear()


def HDArrayShowDeviceInfo(dev=0):
    lib().HDArrayShowDeviceInfo(dev)


_arrays = {}  # handle -> HDArray, for callbacks that receive a handle


def HDArrayCreate(sym, dtype, uA, *sizes):
    s, sp = _i64(sizes)
    h = lib().HDArrayCreatev(sym.encode(), dtype.encode(), _ptr(uA), len(sizes), sp)
    if not h:
        raise HDArrayError(lib().HDArrayGetLastError(), "HDArrayCreate")
    a = HDArray(h, sym, dtype, sizes)
    _arrays[h] = a
    return a


def HDArrayFree(h):
    _chk(lib().HDArrayFree(h), "HDArrayFree")
    _arrays.pop(h.handle if isinstance(h, HDArray) else h, None)


def HDArrayPartition(ptype, sizes, lo, hi, nparts=0):
    dim = len(sizes)
    s, sp = _i64(sizes)
    l, lp = _i64(lo)
    u, up = _i64(hi)
    return _chk(lib().HDArrayPartitionv(ptype, nparts, dim, sp, lp, up), "HDArrayPartition")


def HDArrayPartitionManual(sizes, boxes):
    """boxes: per device (lo, hi) tuples (empty box for a device without work)."""
    dim = len(sizes)
    s, sp = _i64(sizes)
    l, lp = _i64([b[0] for b in boxes])
    u, up = _i64([b[1] for b in boxes])
    return _chk(lib().HDArrayPartitionManual(dim, sp, len(boxes), lp, up), "HDArrayPartitionManual")


def HDArrayApplyKernel(kname, part, *args):
    arrs = [a for a in args if isinstance(a, HDArray)]
    scal = [float(a) for a in args if not isinstance(a, HDArray)]
    A = (_P * max(1, len(arrs)))(*[a.handle for a in arrs])
    S = (ctypes.c_double * max(1, len(scal)))(*scal)
    return _chk(lib().HDArrayApplyKernelv(kname.encode(), part, len(arrs), A, len(scal), S),
                "HDArrayApplyKernel(%s)" % kname)


def HDArrayWrite(h, uA, part):
    return _chk(lib().HDArrayWritev(h, _ptr(uA), part), "HDArrayWrite")


def HDArrayRead(h, uA, part):
    return _chk(lib().HDArrayReadv(h, _ptr(uA), part), "HDArrayRead")


def HDArrayReduce(h, op, part):
    """The double accumulator of HDArrayReduce (HDArrayReduceD)."""
    out = ctypes.c_double()
    _chk(lib().HDArrayReduceD(h, ctypes.byref(out), op, part), "HDArrayReduce")
    return out.value


def HDArraySetAbsoluteUse(kname, part, h, dev, lo, hi):
    l, lp = _i64(lo)
    u, up = _i64(hi)
    return _chk(lib().HDArraySetAbsoluteUsev(kname.encode(), part, h, dev, len(lo), lp, up),
                "HDArraySetAbsoluteUse")


def HDArraySetAbsoluteDef(kname, part, h, dev, lo, hi):
    l, lp = _i64(lo)
    u, up = _i64(hi)
    return _chk(lib().HDArraySetAbsoluteDefv(kname.encode(), part, h, dev, len(lo), lp, up),
                "HDArraySetAbsoluteDef")


def HDArraySetTrapezoidUse(kname, part, h, dev, corners):
    c, cp = _i64(corners)
    return _chk(lib().HDArraySetTrapezoidUsev(kname.encode(), part, h, dev, cp),
                "HDArraySetTrapezoidUse")


def HDArraySetTrapezoidDef(kname, part, h, dev, corners):
    c, cp = _i64(corners)
    return _chk(lib().HDArraySetTrapezoidDefv(kname.encode(), part, h, dev, cp),
                "HDArraySetTrapezoidDef")


def _offs(offs):
    a = np.zeros((len(offs), 3), np.int32)
    for i, o in enumerate(offs):
        a[i, : len(o)] = o
    a = np.ascontiguousarray(a)
    return a, a.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))


def HDArrayRegisterKernel(kname, narr, nscal, space_arg, launcher):
    """Register a user kernel.  launcher(work, scalars, stream) gets a list of HDArrayWork (one per
    logical device with work), the scalars as a list of floats and the cudaStream_t as an int; it
    queues its device work on that stream and returns 0 (or a negative error code)."""
    def thunk(work, nwork, scal, nscal_, stream, user):
        try:
            rc = launcher([work[i] for i in range(nwork)], [scal[i] for i in range(nscal_)], stream or 0)
            return int(rc or 0)
        except Exception:
            return -6  # HDARRAY_ERR_CUDA: the launcher raised
    cb = LAUNCHER(thunk)
    _keep[("kernel", kname)] = cb
    return _chk(lib().HDArrayRegisterKernel(kname.encode(), narr, nscal, space_arg,
                                            ctypes.cast(cb, _P), None), "HDArrayRegisterKernel")


def HDArraySetAllocator(alloc=None, free=None):
    """Device memory from alloc(bytes) -> int pointer and free(int pointer); None, None restores
    cudaMalloc / cudaFree."""
    if alloc is None and free is None:
        return _chk(lib().HDArraySetAllocator(None, None, None), "HDArraySetAllocator")
    a = ALLOC(lambda n, u: int(alloc(int(n)) or 0))
    f = FREE(lambda p, u: free(int(p)))
    _keep.setdefault("allocators", []).append((a, f))  # memory it gave out is freed through it later
    return _chk(lib().HDArraySetAllocator(ctypes.cast(a, _P), ctypes.cast(f, _P), None), "HDArraySetAllocator")


def HDArraySetOffsetUse(kname, arg, offs):
    a, ap = _offs(offs)
    return _chk(lib().HDArraySetOffsetUse(kname.encode(), arg, len(offs), ap), "HDArraySetOffsetUse")


def HDArraySetOffsetDef(kname, arg, offs):
    a, ap = _offs(offs)
    return _chk(lib().HDArraySetOffsetDef(kname.encode(), arg, len(offs), ap), "HDArraySetOffsetDef")


def HDArraySetStream(stream=None):
    """stream: a cudaStream_t as int (e.g. torch.cuda.current_stream().cuda_stream) or None."""
    return _chk(lib().HDArraySetStream(stream), "HDArraySetStream")


def HDArraySetMode(mode):
    return _chk(lib().HDArraySetMode(mode), "HDArraySetMode")


def HDArraySetGemmSplit(parts):
    """HDARRAY_GEMM_BF16X3 (2 bf16 parts per value) or HDARRAY_GEMM_BF16X6 (3 parts)."""
    return _chk(lib().HDArraySetGemmSplit(parts), "HDArraySetGemmSplit")


def HDArraySetAutotune(on=True):
    return _chk(lib().HDArraySetAutotune(1 if on else 0), "HDArraySetAutotune")


def HDArrayBatchBegin():
    return _chk(lib().HDArrayBatchBegin(), "HDArrayBatchBegin")


def HDArrayBatchEnd():
    return _chk(lib().HDArrayBatchEnd(), "HDArrayBatchEnd")


def HDArrayGraphBegin():
    return _chk(lib().HDArrayGraphBegin(), "HDArrayGraphBegin")


def HDArrayGraphEnd():
    gid = ctypes.c_int()
    _chk(lib().HDArrayGraphEnd(ctypes.byref(gid)), "HDArrayGraphEnd")
    return gid.value


def HDArrayGraphLaunch(gid, nrep=1):
    return _chk(lib().HDArrayGraphLaunch(gid, nrep), "HDArrayGraphLaunch")


def HDArrayGraphDestroy(gid):
    return _chk(lib().HDArrayGraphDestroy(gid), "HDArrayGraphDestroy")


def HDArraySync():
    return _chk(lib().HDArraySync(), "HDArraySync")


def HDArrayGetLastError():
    return lib().HDArrayGetLastError()


def HDArrayGetPlan(h):
    """Exchange of the last call that moved h: list of (src, dst, lo(3), hi(3))."""
    n = _chk(lib().HDArrayGetPlan(h, None, 0), "HDArrayGetPlan")
    buf = np.zeros(max(1, n) * 8, np.int64)
    _chk(lib().HDArrayGetPlan(h, buf.ctypes.data_as(_I64P), n), "HDArrayGetPlan")
    out = []
    for i in range(n):
        r = buf[8 * i: 8 * i + 8]
        out.append((int(r[0]), int(r[1]), tuple(int(v) for v in r[2:5]), tuple(int(v) for v in r[5:8])))
    return out


def HDArraySetRankMap(rank_of_dev, my_rank):
    """Logical device d lives on rank rank_of_dev[d]; this process is my_rank.  None: one process."""
    if rank_of_dev is None:
        return _chk(lib().HDArraySetRankMap(0, None, 0), "HDArraySetRankMap")
    r = np.ascontiguousarray(np.asarray(rank_of_dev, dtype=np.int32))
    return _chk(lib().HDArraySetRankMap(len(r), r.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), my_rank),
                "HDArraySetRankMap")


def HDArraySetTransport(fn):
    """fn(array, records, stream) -> int: deliver the cross-rank records (an int64 array of shape
    (n, HDARRAY_RANK_RECORD)) of `array`'s exchange; None removes it."""
    if fn is None:
        _keep.pop("transport", None)
        return _chk(lib().HDArraySetTransport(None, None), "HDArraySetTransport")

    def thunk(h, n, recs, stream, user):
        try:
            r = np.ctypeslib.as_array(recs, shape=(n * HDARRAY_RANK_RECORD,)).reshape(n, HDARRAY_RANK_RECORD).copy()
            return int(fn(_arrays.get(h) or HDArray(h, "?", "?", ()), r, stream or 0) or 0)
        except Exception:
            import traceback
            traceback.print_exc()
            return -6
    cb = TRANSPORT(thunk)
    _keep["transport"] = cb
    return _chk(lib().HDArraySetTransport(ctypes.cast(cb, _P), None), "HDArraySetTransport")


def HDArrayGetRankPlan(h):
    """Cross-rank records of the last call that moved h: int64 array (n, HDARRAY_RANK_RECORD)."""
    n = _chk(lib().HDArrayGetRankPlan(h, None, 0), "HDArrayGetRankPlan")
    buf = np.zeros(max(1, n) * HDARRAY_RANK_RECORD, np.int64)
    _chk(lib().HDArrayGetRankPlan(h, buf.ctypes.data_as(_I64P), n), "HDArrayGetRankPlan")
    return buf[: n * HDARRAY_RANK_RECORD].reshape(n, HDARRAY_RANK_RECORD)


def HDArrayStagingBytes(h, recs):
    r, rp = _i64(recs)
    return _chk(lib().HDArrayStagingBytes(h, len(r) // HDARRAY_RANK_RECORD, rp), "HDArrayStagingBytes")


def HDArrayPackBoxes(h, recs, staging, nbytes):
    r, rp = _i64(recs)
    return _chk(lib().HDArrayPackBoxes(h, len(r) // HDARRAY_RANK_RECORD, rp, _ptr(staging), nbytes),
                "HDArrayPackBoxes")


def HDArrayUnpackBoxes(h, recs, staging, nbytes):
    r, rp = _i64(recs)
    return _chk(lib().HDArrayUnpackBoxes(h, len(r) // HDARRAY_RANK_RECORD, rp, _ptr(staging), nbytes),
                "HDArrayUnpackBoxes")


def HDArrayGetGDEF(h, p, q):
    n = _chk(lib().HDArrayGetGDEF(h, p, q, None, 0), "HDArrayGetGDEF")
    buf = np.zeros(max(1, n) * 6, np.int64)
    _chk(lib().HDArrayGetGDEF(h, p, q, buf.ctypes.data_as(_I64P), n), "HDArrayGetGDEF")
    return [(tuple(int(v) for v in buf[6 * i: 6 * i + 3]), tuple(int(v) for v in buf[6 * i + 3: 6 * i + 6]))
            for i in range(n)]


def HDArrayGetDeviceBuffer(h, dev):
    """(device pointer or None, alloc lo (3), alloc hi (3), element strides (3))."""
    p = _P()
    lo = np.zeros(3, np.int64)
    hi = np.zeros(3, np.int64)
    st = np.zeros(3, np.int64)
    _chk(lib().HDArrayGetDeviceBuffer(h, dev, ctypes.byref(p), lo.ctypes.data_as(_I64P),
                                      hi.ctypes.data_as(_I64P), st.ctypes.data_as(_I64P)),
         "HDArrayGetDeviceBuffer")
    return p.value, tuple(int(v) for v in lo), tuple(int(v) for v in hi), tuple(int(v) for v in st)


def HDArrayReadDeviceBuffer(h, dev, lo, hi, out):
    """Raw contents of box [lo, hi) of device dev's buffer into the dense array `out`."""
    l, lp = _i64(lo)
    u, up = _i64(hi)
    return _chk(lib().HDArrayReadDeviceBuffer(h, dev, lp, up, _ptr(out)), "HDArrayReadDeviceBuffer")


def HDArrayReduceBufferNoAlloc(x, dtype, extent, strides, op, result, stream=None):
    """Allocation-free reduction of a strided device box into the device double `result`."""
    e, ep = _i64(extent)
    s, sp = _i64(strides)
    return _chk(lib().HDArrayReduceBufferNoAlloc(_ptr(x), dtype.encode(), len(extent), ep, sp, op,
                                                 _ptr(result), stream), "HDArrayReduceBufferNoAlloc")


def HDArrayGetCounters():
    """dict: launches, bytes_moved, plans, plan_hits, graph_launches."""
    buf = np.zeros(5, np.int64)
    _chk(lib().HDArrayGetCounters(buf.ctypes.data_as(_I64P), 5), "HDArrayGetCounters")
    return dict(zip(["launches", "bytes_moved", "plans", "plan_hits", "graph_launches"],
                    (int(v) for v in buf)))
