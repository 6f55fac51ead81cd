"""Python driver for the plain C oracle of the HDArray hot path.

TEST INFRASTRUCTURE. Only tests/, the smoke check and the CPU-baseline leg of bench.py import
this module. It shares no code with the GPU library: it keeps its own kernel table (the use/def
offsets of each built-in kernel, read from the paper), its own partition and section
definitions (in hdarray_oracle.c), and evaluates everything on one unpartitioned array.

The program interface mirrors the HDArray calls of Table 2 (Sec. 3.1):
``create``, ``partition`` / ``partition_manual``, ``write``, ``apply`` (HDArrayApplyKernel),
``read``, ``reduce``, ``set_absolute_use/def`` and ``set_trapezoid_use/def``.  Each call that
moves data returns the messages of Eq. 1-2 as computed by the per-element state machine.

Two array modes:
  * full arrays: every element is tracked and the global values G are kept (numpy);
  * sampled arrays (``coords`` given): only the listed elements are tracked, sets only, no values.
    Membership of each listed element in every section is decided by the same predicates, so the
    messages involving those elements are exact at any array size.
"""
import ctypes
import os

import numpy as np

from . import build as _build

ALL = -(2 ** 31)  # the '*' offset component (Sec. 3, offset clauses)

ROW, COL, BLOCK = 0, 1, 2
SUM, PROD, MAX, MIN = 0, 1, 2, 3
PREC = {"double": 0, "float": 1, "bf16": 2}
NPDTYPE = {"double": np.float64, "float": np.float32, "bf16": np.uint16}

_lib = None


def lib():
    """Load (building first if needed) the oracle shared library."""
    global _lib
    if _lib is None:
        path = _build.build()
        L = ctypes.CDLL(path)
        P = ctypes.c_void_p
        i64, i32 = ctypes.c_int64, ctypes.c_int
        sig = {
            "orc_partition_box": (i32, [i32, i32, i32, i32, P, P, P, P]),
            "orc_mask_box": (None, [P, P, P, P]),
            "orc_mask_offsets": (None, [P, P, P, i32, P, P]),
            "orc_mask_trapezoid": (i32, [P, P, P]),
            "orc_pred_box": (None, [P, P, i64, P, P]),
            "orc_pred_offsets": (None, [P, P, P, i32, P, i64, P, P]),
            "orc_pred_trapezoid": (i32, [P, i64, P, P]),
            "orc_state_new": (P, [i64, i32]),
            "orc_state_free": (None, [P]),
            "orc_state_use": (i64, [P, P, P, P]),
            "orc_state_def": (i32, [P, P]),
            "orc_state_get": (None, [P, P, P]),
            "orc_state_sgdef": (None, [P, i32, i32, P]),
            "orc_f32_to_bf16_array": (None, [i64, P, P]),
            "orc_bf16_to_f32_array": (None, [i64, P, P]),
            "orc_jacobi2d": (i32, [i32, i64, i64, P, P, P]),
            "orc_stencil3d": (i32, [i32, i64, i64, i64, P, P, P]),
            "orc_conv2d": (i32, [i32, i64, i64, P, P, P, P]),
            "orc_colmean": (i32, [i32, i64, i64, P, P, P]),
            "orc_center": (i32, [i32, i64, i64, P, P, P, P]),
            "orc_syrk_upper": (i32, [i32, i64, i64, ctypes.c_double, P, P, P]),
            "orc_colnorm": (i32, [i32, i64, i64, P, P, P]),
            "orc_colscale": (i32, [i32, i64, i64, P, P, P, P]),
            "orc_symmetrize": (i32, [i32, i64, P, P]),
            "orc_copy": (None, [i32, i64, P, P, P]),
            "orc_sqdiff": (None, [i32, i64, P, P, P, P]),
            "orc_gemm": (None, [i64, i64, i64, ctypes.c_double, ctypes.c_double, P, P, P, P]),
            "orc_gemm_entries": (None, [i64, i64, ctypes.c_double, ctypes.c_double, P, P, P,
                                        i64, P, P]),
            "orc_reduce": (i32, [i32, i64, P, P, i32, P]),
            "orc_set_threads": (i32, [i32]),
        }
        for name, (res, args) in sig.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def set_threads(n):
    """Threads of the stencil value loops (same results with any count); returns the count used
    (1 when the oracle was built without OpenMP)."""
    return lib().orc_set_threads(int(n))


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p) if a is not None else None


def _i64(seq):
    return np.ascontiguousarray(np.asarray(seq, dtype=np.int64))


def _dims3(dims):
    """Extents padded to three dimensions (unused dimensions have extent 1)."""
    d = list(dims) + [1] * (3 - len(dims))
    return _i64(d)


def _lo3(lo):
    """Lower corner padded to three dimensions (coordinate 0)."""
    return _i64(list(lo) + [0] * (3 - len(lo)))


def _hi3(hi):
    """Upper corner padded to three dimensions (exclusive bound 1)."""
    return _i64(list(hi) + [1] * (3 - len(hi)))


def _off3(offs):
    out = []
    for o in offs:
        o = list(o) + [0] * (3 - len(o))
        out.append(o)
    return np.ascontiguousarray(np.asarray(out, dtype=np.int32).reshape(-1, 3))


# --------------------------------------------------------------------------------------------
# Element-level helpers
# --------------------------------------------------------------------------------------------

def f32_to_bf16(x):
    x = np.ascontiguousarray(np.asarray(x, dtype=np.float32))
    out = np.empty(x.shape, dtype=np.uint16)
    lib().orc_f32_to_bf16_array(x.size, _p(x), _p(out))
    return out


def bf16_to_f32(h):
    h = np.ascontiguousarray(np.asarray(h, dtype=np.uint16))
    out = np.empty(h.shape, dtype=np.float32)
    lib().orc_bf16_to_f32_array(h.size, _p(h), _p(out))
    return out


def partition_boxes(ptype, nparts, dims, lo, hi):
    """Work boxes of an even ROW/COL/BLOCK partition (HDArrayPartition, Sec. 3.1)."""
    dim = len(dims)
    rlo, rhi = _lo3(lo), _hi3(hi)
    boxes = []
    for p in range(nparts):
        blo, bhi = np.zeros(3, np.int64), np.zeros(3, np.int64)
        rc = lib().orc_partition_box(ptype, nparts, p, dim, _p(rlo), _p(rhi), _p(blo), _p(bhi))
        if rc != 0:
            raise ValueError("invalid partition request")
        boxes.append((tuple(int(v) for v in blo), tuple(int(v) for v in bhi)))
    return boxes


def gemm_entries(A, B, C, alpha, beta, ij):
    """New C[i][j] of Listing 3 (binary64) for the listed (i, j) only."""
    A = np.ascontiguousarray(A, dtype=np.float64)
    B = np.ascontiguousarray(B, dtype=np.float64)
    ij = np.ascontiguousarray(np.asarray(ij, dtype=np.int64).reshape(-1, 2))
    nk, nj = B.shape
    Cc = None if C is None else np.ascontiguousarray(C, dtype=np.float64)
    out = np.empty(len(ij), np.float64)
    lib().orc_gemm_entries(nj, nk, alpha, beta, _p(A), _p(B), _p(Cc), len(ij), _p(ij), _p(out))
    return out


# --------------------------------------------------------------------------------------------
# Built-in kernel table: which elements each argument uses and defines, as offsets relative to
# a work item (Sec. 3, offset clauses), and what the kernel computes.
# --------------------------------------------------------------------------------------------

class KernelSpec:
    def __init__(self, narr, use, defs, run, nscal=0):
        self.narr = narr
        self.use = use      # {arg index: [offset, ...]}
        self.defs = defs    # {arg index: [offset, ...]}
        self.run = run      # run(oracle, arrays, work_mask_over_index_space, scalars)
        self.nscal = nscal


def _run_jacobi2d(o, arrs, work, scal):
    X, Y = arrs
    rc = lib().orc_jacobi2d(X.prec, X.dims[0], X.dims[1], _p(X.G), _p(Y.G), _p(work))
    if rc != 0:
        raise ValueError("jacobi2d: work element on the array border")


def _run_conv2d(o, arrs, work, scal):
    X, Y = arrs
    w = np.ascontiguousarray(np.array(scal, dtype=np.float64))
    if w.size != 9:
        raise ValueError("conv2d: nine weights")
    rc = lib().orc_conv2d(X.prec, X.dims[0], X.dims[1], _p(X.G), _p(Y.G), _p(work), _p(w))
    if rc != 0:
        raise ValueError("conv2d: work element on the array border")


def _run_colmean(o, arrs, work, scal):
    X, M = arrs
    if lib().orc_colmean(X.prec, X.dims[0], X.dims[1], _p(X.G), _p(M.G), _p(work)) != 0:
        raise ValueError("colmean: double or float arrays")


def _run_center(o, arrs, work, scal):
    X, M, Xc = arrs
    if lib().orc_center(X.prec, X.dims[0], X.dims[1], _p(X.G), _p(M.G), _p(Xc.G), _p(work)) != 0:
        raise ValueError("center: double or float arrays")


def _run_colnorm(o, arrs, work, scal):
    X, S = arrs
    if lib().orc_colnorm(X.prec, X.dims[0], X.dims[1], _p(X.G), _p(S.G), _p(work)) != 0:
        raise ValueError("colnorm: double or float arrays")


def _run_colscale(o, arrs, work, scal):
    X, S, Y = arrs
    if lib().orc_colscale(X.prec, X.dims[0], X.dims[1], _p(X.G), _p(S.G), _p(Y.G), _p(work)) != 0:
        raise ValueError("colscale: double or float arrays")


def _run_syrk(o, arrs, work, scal):
    X, C = arrs
    if lib().orc_syrk_upper(X.prec, X.dims[0], X.dims[1], float(scal[0]), _p(X.G), _p(C.G), _p(work)) != 0:
        raise ValueError("syrk: double or float arrays")


def _run_symmetrize(o, arrs, work, scal):
    (C,) = arrs
    lib().orc_symmetrize(C.prec, C.dims[0], _p(C.G), _p(work))


def _run_stencil3d(o, arrs, work, scal):
    X, Y = arrs
    rc = lib().orc_stencil3d(X.prec, X.dims[0], X.dims[1], X.dims[2], _p(X.G), _p(Y.G), _p(work))
    if rc != 0:
        raise ValueError("stencil3d: work element on the array border")


def _run_copy(o, arrs, work, scal):
    X, Y = arrs
    lib().orc_copy(X.prec, X.total, _p(X.G), _p(Y.G), _p(work))


def _run_sqdiff(o, arrs, work, scal):
    X, Y, R = arrs
    if R.prec != 0:
        raise ValueError("sqdiff: residual array must be double")
    lib().orc_sqdiff(X.prec, X.total, _p(X.G), _p(Y.G), _p(R.G), _p(work))


def _run_gemm(o, arrs, work, scal):
    A, B, C = arrs
    alpha, beta = scal[0], scal[1]
    ni, nk = A.dims[0], A.dims[1]
    nj = B.dims[1]
    if A.prec == 0:
        lib().orc_gemm(ni, nj, nk, alpha, beta, _p(A.G), _p(B.G), _p(C.G), _p(work))
    else:
        # binary32 storage: the reference result is the binary64 product of the stored inputs,
        # rounded once to the storage type.
        A64 = np.ascontiguousarray(A.values64())
        B64 = np.ascontiguousarray(B.values64())
        C64 = np.ascontiguousarray(C.values64())
        lib().orc_gemm(ni, nj, nk, alpha, beta, _p(A64), _p(B64), _p(C64), _p(work))
        C.G[...] = C64.astype(np.float32).reshape(C.G.shape)


_J2 = [(0, -1), (0, 1), (-1, 0), (1, 0)]
_S3 = [(0, 0, -1), (0, 0, 1), (0, -1, 0), (0, 1, 0), (-1, 0, 0), (1, 0, 0)]
_C2 = _J2 + [(-1, -1), (-1, 1), (1, -1), (1, 1)]

KERNELS = {
    # Sec. 5, Jacobi kernel 1: use B at four offsets, define A at (0, 0).  Arguments (B, A).
    "jacobi2d": KernelSpec(2, {0: _J2}, {1: [(0, 0)]}, _run_jacobi2d),
    # Sec. 5, Jacobi kernel 2 (B = A): zero offsets.  Arguments (A, B).
    "copy": KernelSpec(2, {0: [(0, 0, 0)]}, {1: [(0, 0, 0)]}, _run_copy),
    # 3-D 7-point analogue of kernel 1.  Arguments (B, A).
    "stencil3d": KernelSpec(2, {0: _S3}, {1: [(0, 0, 0)]}, _run_stencil3d),
    # Residual field R = (X - Y)^2, zero offsets.  Arguments (X, Y, R).
    "sqdiff": KernelSpec(3, {0: [(0, 0, 0)], 1: [(0, 0, 0)]}, {2: [(0, 0, 0)]}, _run_sqdiff),
    # Listing 3: use(A,(0,*)) use(B,(*,0)) def(C,(0,0)); work items are the (i, j) of C.
    "gemm": KernelSpec(3, {0: [(0, ALL)], 1: [(ALL, 0)]}, {2: [(0, 0)]}, _run_gemm, nscal=2),
    # The same contraction with A lower triangular; its use of A is normally given as trapezoids.
    "trmm": KernelSpec(3, {0: [(0, ALL)], 1: [(ALL, 0)]}, {2: [(0, 0)]}, _run_gemm, nscal=2),
    # The communication step alone (use at zero offsets or absolute sections, no definition).
    "exchange": KernelSpec(1, {0: [(0, 0, 0)]}, {}, None),
    # Sec. 5, 2-D convolution: the Jacobi offsets plus the four diagonals and the centre, nine
    # weights as scalars.  Arguments (X, Y, w0 .. w8).
    "conv2d": KernelSpec(2, {0: _C2 + [(0, 0)]}, {1: [(0, 0)]}, _run_conv2d, nscal=9),
    # Covariance (Sec. 5.1).  Column means of X (n x m) into M (1 x m): use X's whole column.
    "colmean": KernelSpec(2, {0: [(ALL, 0)]}, {1: [(0, 0)]}, _run_colmean),
    # Xc = X - M (M broadcast down the columns).  Arguments (X, M, Xc).
    "center": KernelSpec(3, {0: [(0, 0)], 1: [(ALL, 0)]}, {2: [(0, 0)]}, _run_center),
    # Correlation: column norms S (1 x m) of X, and Y = X / S (S broadcast down the columns).
    "colnorm": KernelSpec(2, {0: [(ALL, 0)]}, {1: [(0, 0)]}, _run_colnorm),
    "colscale": KernelSpec(3, {0: [(0, 0)], 1: [(ALL, 0)]}, {2: [(0, 0)]}, _run_colscale),
    # C[i][j] = alpha * (X^T X)[i][j] for j >= i.  Arguments (X, C, alpha).  The use of X (columns i
    # and j of every row) is not an offset pattern: by default all of X, normally narrowed with
    # absolute sections; the definition is normally narrowed to the upper trapezoid.
    "syrk": KernelSpec(2, {0: [(ALL, ALL)]}, {1: [(0, 0)]}, _run_syrk, nscal=1),
    # C[i][j] = C[j][i] for j < i (the transposed use likewise narrowed with absolute sections,
    # the definition to the lower trapezoid).  Argument (C).
    "symmetrize": KernelSpec(1, {0: [(ALL, ALL)]}, {0: [(0, 0)]}, _run_symmetrize),
}


# --------------------------------------------------------------------------------------------
# Arrays and the program driver
# --------------------------------------------------------------------------------------------

class OArray:
    def __init__(self, name, dtype, dims, P, coords=None):
        self.name = name
        self.dtype = dtype
        self.prec = PREC[dtype]
        self.dims = tuple(int(d) for d in dims)
        self.n3 = _dims3(self.dims)
        self.coords = None
        if coords is not None:
            c = np.zeros((len(coords), 3), np.int64)
            cc = np.asarray(coords, dtype=np.int64).reshape(len(coords), -1)
            c[:, : cc.shape[1]] = cc
            self.coords = np.ascontiguousarray(c)
            self.total = len(coords)
            self.G = None
        else:
            self.total = int(np.prod(self.dims))
            self.G = np.zeros(self.dims, dtype=NPDTYPE[dtype])  # Create: zero, nothing copied
        self.P = P
        self.state = lib().orc_state_new(self.total, P)
        if not self.state:
            raise MemoryError("oracle state")

    def __del__(self):
        try:
            if self.state:
                lib().orc_state_free(self.state)
                self.state = None
        except Exception:
            pass

    def values64(self):
        if self.prec == 2:
            return bf16_to_f32(self.G).astype(np.float64)
        return self.G.astype(np.float64)

    # section masks over this array's tracked elements ---------------------------------------
    def mask_box(self, lo, hi, out):
        lo3, hi3 = _lo3(lo), _hi3(hi)
        if self.coords is None:
            lib().orc_mask_box(_p(self.n3), _p(lo3), _p(hi3), _p(out))
        else:
            lib().orc_pred_box(_p(lo3), _p(hi3), self.total, _p(self.coords), _p(out))

    def mask_offsets(self, wlo, whi, offs, out):
        wlo3, whi3 = _lo3(wlo), _hi3(whi)
        o = _off3(offs)
        if self.coords is None:
            lib().orc_mask_offsets(_p(self.n3), _p(wlo3), _p(whi3), len(o), _p(o), _p(out))
        else:
            lib().orc_pred_offsets(_p(self.n3), _p(wlo3), _p(whi3), len(o), _p(o), self.total,
                                   _p(self.coords), _p(out))

    def mask_trapezoid(self, corners, out):
        c = _i64(corners)
        if self.coords is None:
            rc = lib().orc_mask_trapezoid(_p(self.n3), _p(c), _p(out))
        else:
            rc = lib().orc_pred_trapezoid(_p(c), self.total, _p(self.coords), _p(out))
        if rc != 0:
            raise ValueError("invalid trapezoid corners")

    def state_get(self):
        owner = np.empty(self.total, np.int16)
        have = np.empty((self.P, self.total), np.uint8)
        lib().orc_state_get(self.state, _p(owner), _p(have))
        return owner, have

    def sgdef(self, p, q):
        m = np.empty(self.total, np.uint8)
        lib().orc_state_sgdef(self.state, p, q, _p(m))
        return m


class Messages:
    """Messages of one call for one array: src[p, e] = sending device (or -1), counts[q, p]."""

    def __init__(self, src, counts):
        self.src = src
        self.counts = counts

    def elements(self, q, p):
        return np.nonzero(self.src[p] == q)[0]

    @property
    def total(self):
        return int(self.counts.sum())


class Oracle:
    """Whole-array HDArray program with per-element communication bookkeeping."""

    def __init__(self, ndev):
        self.ndev = ndev
        self.arrays = []
        self.abs_use = {}   # (kname, part_id, array id, dev) -> list of shapes
        self.abs_def = {}
        self.parts = []

    # Table 2: HDArrayCreate ---------------------------------------------------------------
    def create(self, name, dtype, dims, coords=None):
        a = OArray(name, dtype, dims, self.ndev, coords)
        self.arrays.append(a)
        return a

    # Table 2: HDArrayPartition (even split) and the partition clause (manual regions) -------
    def partition(self, ptype, dims, lo, hi, nparts=None):
        P = self.ndev if nparts is None else nparts
        if P > self.ndev:
            raise ValueError("more parts than devices")
        boxes = partition_boxes(ptype, P, dims, lo, hi)
        self.parts.append(boxes + [None] * (self.ndev - P))
        return len(self.parts) - 1

    def partition_manual(self, boxes):
        """boxes[p] = (lo, hi) of device p, or None for a device without work."""
        if len(boxes) > self.ndev:
            raise ValueError("more parts than devices")
        b = []
        for x in boxes:
            if x is None:
                b.append(None)
            else:
                lo, hi = x
                b.append((tuple(lo) + (0,) * (3 - len(lo)), tuple(hi) + (1,) * (3 - len(hi))))
        self.parts.append(b + [None] * (self.ndev - len(b)))
        return len(self.parts) - 1

    # Table 2: absolute sections and trapezoids -------------------------------------------
    def set_absolute_use(self, kname, part, arr, dev, lo, hi):
        self.abs_use.setdefault((kname, part, id(arr)), {}).setdefault(dev, []).append(("box", lo, hi))

    def set_absolute_def(self, kname, part, arr, dev, lo, hi):
        self.abs_def.setdefault((kname, part, id(arr)), {}).setdefault(dev, []).append(("box", lo, hi))

    def set_trapezoid_use(self, kname, part, arr, dev, corners):
        self.abs_use.setdefault((kname, part, id(arr)), {}).setdefault(dev, []).append(("trap", corners))

    def set_trapezoid_def(self, kname, part, arr, dev, corners):
        self.abs_def.setdefault((kname, part, id(arr)), {}).setdefault(dev, []).append(("trap", corners))

    # masks ------------------------------------------------------------------------------
    def _region_masks(self, arr, part):
        m = np.zeros((self.ndev, arr.total), np.uint8)
        for p, box in enumerate(self.parts[part]):
            if box is not None:
                arr.mask_box(box[0], box[1], m[p])
        return m

    def _clause_masks(self, arr, part, offsets, absolute):
        m = np.zeros((self.ndev, arr.total), np.uint8)
        if absolute is not None:
            for dev, shapes in absolute.items():
                for s in shapes:
                    if s[0] == "box":
                        arr.mask_box(s[1], s[2], m[dev])
                    else:
                        arr.mask_trapezoid(s[1], m[dev])
            return m
        if offsets:
            for p, box in enumerate(self.parts[part]):
                if box is not None:
                    arr.mask_offsets(box[0], box[1], offsets, m[p])
        return m

    def _use(self, arr, use_mask):
        src = np.empty((self.ndev, arr.total), np.int16)
        counts = np.zeros((self.ndev, self.ndev), np.int64)
        n = lib().orc_state_use(arr.state, _p(np.ascontiguousarray(use_mask)), _p(src), _p(counts))
        if n < 0:
            raise RuntimeError("oracle: element missing on every device")
        return Messages(src, counts)

    def _def(self, arr, def_mask):
        rc = lib().orc_state_def(arr.state, _p(np.ascontiguousarray(def_mask)))
        if rc == -2:
            raise ValueError("race: two devices define the same element")

    # Table 2: HDArrayWrite -- user array into the devices of a partition (a definition) ----
    def write(self, arr, values, part):
        reg = self._region_masks(arr, part)
        if arr.G is not None and values is not None:
            v = np.asarray(values).reshape(arr.dims)
            sel = reg.any(axis=0).reshape(arr.dims).astype(bool)
            arr.G[sel] = v.astype(arr.G.dtype)[sel]
        self._def(arr, reg)

    # Table 2: HDArrayRead -- each device's region back to the user (a use of the region) ----
    def read(self, arr, part):
        reg = self._region_masks(arr, part)
        msgs = self._use(arr, reg)
        return msgs

    # Table 2: HDArrayReduce -- fold the partition's regions (a use of the regions) ---------
    def reduce(self, arr, op, part):
        reg = self._region_masks(arr, part)
        if (reg.sum(axis=0) > 1).any():
            raise ValueError("reduce over overlapping regions")
        msgs = self._use(arr, reg)
        out = ctypes.c_double()
        union = np.ascontiguousarray(reg.any(axis=0).astype(np.uint8))
        rc = lib().orc_reduce(arr.prec, arr.total, _p(np.ascontiguousarray(arr.G)), _p(union), op,
                              ctypes.byref(out))
        if rc != 0:
            raise ValueError("unknown reduce op")
        return out.value, msgs

    # Table 2: HDArrayApplyKernel -- messages (Eq. 1-2), compute, definitions (Eq. 3-4) ------
    def apply(self, kname, part, arrays, scalars=(), compute=True):
        k = KERNELS[kname]
        if len(arrays) != k.narr:
            raise ValueError("wrong number of array arguments")
        uses, defs = {}, {}
        for i, a in enumerate(arrays):
            au = self.abs_use.get((kname, part, id(a)))
            ad = self.abs_def.get((kname, part, id(a)))
            u = self._clause_masks(a, part, k.use.get(i), au)
            d = self._clause_masks(a, part, k.defs.get(i), ad)
            if id(a) in uses:
                uses[id(a)] = (a, uses[id(a)][1] | u)
                defs[id(a)] = (a, defs[id(a)][1] | d)
            else:
                uses[id(a)] = (a, u)
                defs[id(a)] = (a, d)
        msgs = {}
        for key, (a, u) in uses.items():
            msgs[key] = self._use(a, u)
        if compute and k.run is not None and all(a.G is not None for a in arrays):
            space = arrays[-1]  # the defined array spans the work-item index space
            work = np.zeros(space.total, np.uint8)
            for box in self.parts[part]:
                if box is not None:
                    space.mask_box(box[0], box[1], work)
            k.run(self, arrays, work, scalars)
        for key, (a, d) in defs.items():
            self._def(a, d)
        return {i: msgs[id(a)] for i, a in enumerate(arrays)}
