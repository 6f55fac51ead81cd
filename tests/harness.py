"""Test harness: run one HDArray program on the oracle and on the library, compare.

A program is a list of operations:
  ("create", name, dtype, dims)
  ("part", name, ptype, dims, lo, hi[, nparts])    even ROW/COL/BLOCK partition of a region
  ("manual", name, dims, boxes)                    partition clause: (lo, hi) per device
  ("write", array, part[, values])
  ("apply", kernel, part, [arrays...], [scalars...])
  ("read", array, part)
  ("reduce", array, op, part)
  ("offset_use", kernel, arg, offsets)             replace a kernel's use offsets
  ("abs_use" | "abs_def", kernel, part, array, dev, lo, hi)
  ("trap_use" | "trap_def", kernel, part, array, dev, corners)

The oracle computes messages element by element; the library's exchange of each call is read
back with HDArrayGetPlan and rasterised.  Both sides get the same seeded inputs.
"""
import copy

import numpy as np

import oracle
from oracle import Oracle


def _flat_index(dims, lo, hi):
    """Flat row-major indices of a box (user order, padded to 3-D)."""
    n = list(dims) + [1] * (3 - len(dims))
    r = [np.arange(lo[d], hi[d]) for d in range(3)]
    g = np.meshgrid(*r, indexing="ij")
    return (g[0] * n[1] * n[2] + g[1] * n[2] + g[2]).ravel()


class OracleRun:
    """Runs a program on the oracle; messages per op as {array name: Messages}."""

    def __init__(self, ndev, coords=None):
        self.o = Oracle(ndev)
        self.o_kernels = {k: copy.copy(v) for k, v in oracle.KERNELS.items()}
        self.coords = coords or {}
        self.arrays, self.parts = {}, {}

    def run(self, prog, values=None):
        out = []
        values = values or {}
        for op in prog:
            out.append(self.step(op, values))
        return out

    def step(self, op, values):
        o = self.o
        kind = op[0]
        if kind == "create":
            _, name, dtype, dims = op
            self.arrays[name] = o.create(name, dtype, dims, coords=self.coords.get(name))
            return None
        if kind == "part":
            name, ptype, dims, lo, hi = op[1:6]
            nparts = op[6] if len(op) > 6 else None
            self.parts[name] = o.partition(ptype, dims, lo, hi, nparts)
            return None
        if kind == "manual":
            self.parts[op[1]] = o.partition_manual(op[3])
            return None
        if kind == "write":
            a = self.arrays[op[1]]
            v = values.get(op[1]) if len(op) < 4 else op[3]
            o.write(a, v, self.parts[op[2]])
            return None
        if kind == "apply":
            _, kname, part, names = op[:4]
            scal = op[4] if len(op) > 4 else ()
            spec = self.o_kernels[kname]
            saved = oracle.KERNELS[kname]
            oracle.KERNELS[kname] = spec
            try:
                msgs = o.apply(kname, self.parts[part], [self.arrays[n] for n in names], scal,
                               compute=all(self.arrays[n].G is not None for n in names))
            finally:
                oracle.KERNELS[kname] = saved
            res = {}
            for i, n in enumerate(names):
                if i in spec.use or (kname, self.parts[part], id(self.arrays[n])) in o.abs_use:
                    res[n] = msgs[i]
            return res
        if kind == "read":
            return {op[1]: o.read(self.arrays[op[1]], self.parts[op[2]])}
        if kind == "reduce":
            val, msgs = o.reduce(self.arrays[op[1]], op[2], self.parts[op[3]])
            return {op[1]: msgs, "_value": val}
        if kind == "offset_use":
            _, kname, arg, offs = op
            spec = copy.copy(self.o_kernels[kname])
            spec.use = dict(spec.use)
            spec.use[arg] = [tuple(x) for x in offs]
            self.o_kernels[kname] = spec
            return None
        if kind in ("abs_use", "abs_def"):
            _, kname, part, name, dev, lo, hi = op
            f = o.set_absolute_use if kind == "abs_use" else o.set_absolute_def
            f(kname, self.parts[part], self.arrays[name], dev, lo, hi)
            return None
        if kind in ("trap_use", "trap_def"):
            _, kname, part, name, dev, corners = op
            f = o.set_trapezoid_use if kind == "trap_use" else o.set_trapezoid_def
            f(kname, self.parts[part], self.arrays[name], dev, corners)
            return None
        raise ValueError(kind)


class LibraryRun:
    """Runs a program on libhdarray.so; messages per op as {array name: [(src, dst, lo, hi)]}."""

    def __init__(self, H, ndev):
        self.H = H
        self.ndev = ndev
        self.arrays, self.parts, self.dims = {}, {}, {}
        self.kernel_use = {}

    def run(self, prog, values=None):
        return [self.step(op, values or {}) for op in prog]

    def step(self, op, values):
        H = self.H
        kind = op[0]
        if kind == "create":
            _, name, dtype, dims = op
            self.arrays[name] = H.HDArrayCreate(name, dtype, None, *dims)
            self.dims[name] = tuple(dims)
            return None
        if kind == "part":
            name, ptype, dims, lo, hi = op[1:6]
            nparts = op[6] if len(op) > 6 else self.ndev
            self.parts[name] = H.HDArrayPartition(ptype, dims, lo, hi, nparts)
            return None
        if kind == "manual":
            dims, boxes = op[2], op[3]
            dim = len(dims)
            bx = [b if b is not None else ((0,) * dim, (0,) * dim) for b in boxes]
            self.parts[op[1]] = H.HDArrayPartitionManual(dims, bx)
            return None
        if kind == "write":
            v = values.get(op[1]) if len(op) < 4 else op[3]
            H.HDArrayWrite(self.arrays[op[1]], v, self.parts[op[2]])
            return None
        if kind == "apply":
            _, kname, part, names = op[:4]
            scal = op[4] if len(op) > 4 else ()
            H.HDArrayApplyKernel(kname, self.parts[part], *[self.arrays[n] for n in names], *scal)
            used = self.used_args(kname, part, names)
            return {n: H.HDArrayGetPlan(self.arrays[n]) for n in used}
        if kind == "read":
            H.HDArrayRead(self.arrays[op[1]], values.get("_read_" + op[1]), self.parts[op[2]])
            return {op[1]: H.HDArrayGetPlan(self.arrays[op[1]])}
        if kind == "reduce":
            val = H.HDArrayReduce(self.arrays[op[1]], op[2], self.parts[op[3]])
            return {op[1]: H.HDArrayGetPlan(self.arrays[op[1]]), "_value": val}
        if kind == "offset_use":
            _, kname, arg, offs = op
            H.HDArraySetOffsetUse(kname, arg, offs)
            self.kernel_use[(kname, arg)] = offs
            return None
        if kind in ("abs_use", "abs_def"):
            _, kname, part, name, dev, lo, hi = op
            f = H.HDArraySetAbsoluteUse if kind == "abs_use" else H.HDArraySetAbsoluteDef
            f(kname, self.parts[part], self.arrays[name], dev, lo, hi)
            if kind == "abs_use":
                self.kernel_use[(kname, part, name)] = True
            return None
        if kind in ("trap_use", "trap_def"):
            _, kname, part, name, dev, corners = op
            f = H.HDArraySetTrapezoidUse if kind == "trap_use" else H.HDArraySetTrapezoidDef
            f(kname, self.parts[part], self.arrays[name], dev, corners)
            if kind == "trap_use":
                self.kernel_use[(kname, part, name)] = True
            return None
        raise ValueError(kind)

    def used_args(self, kname, part, names):
        spec = oracle.KERNELS[kname]
        used = []
        for i, n in enumerate(names):
            if i in spec.use or (kname, i) in self.kernel_use or (kname, part, n) in self.kernel_use:
                if n not in used:
                    used.append(n)
        return used


def rasterise(moves, dims, ndev):
    """Library moves -> src[p, e] (-1 where nothing arrives); fails on overlapping boxes."""
    total = int(np.prod(dims))
    src = np.full((ndev, total), -1, np.int32)
    for q, p, lo, hi in moves:
        idx = _flat_index(dims, lo, hi)
        assert (src[p, idx] == -1).all(), "overlapping moves"
        src[p, idx] = q
    return src


def moves_at(moves, ndev, coords):
    """Library moves evaluated at listed coordinates: src[p, i]."""
    c = np.zeros((len(coords), 3), np.int64)
    cc = np.asarray(coords, np.int64).reshape(len(coords), -1)
    c[:, : cc.shape[1]] = cc
    src = np.full((ndev, len(coords)), -1, np.int32)
    for q, p, lo, hi in moves:
        inside = np.ones(len(coords), bool)
        for d in range(3):
            inside &= (c[:, d] >= lo[d]) & (c[:, d] < hi[d])
        assert (src[p, inside] == -1).all(), "overlapping moves"
        src[p, inside] = q
    return src


def compare_messages(orc_out, lib_out, prog, dims_of, ndev, coords=None):
    """Assert the library's exchange equals the oracle's messages for every op."""
    ncalls = 0
    for op, om, lm in zip(prog, orc_out, lib_out):
        if om is None:
            continue
        for name, msgs in om.items():
            if name.startswith("_"):
                continue
            assert name in lm, (op, name)
            if coords and name in coords:
                got = moves_at(lm[name], ndev, coords[name])
            else:
                got = rasterise(lm[name], dims_of[name], ndev)
            want = msgs.src.astype(np.int32)
            assert want.shape == got.shape
            if not np.array_equal(want, got):
                bad = np.argwhere(want != got)[:5]
                raise AssertionError("messages differ at %s for %s: (dev, elem) %s oracle %s library %s"
                                     % (op, name, bad.tolist(), [want[tuple(b)] for b in bad],
                                        [got[tuple(b)] for b in bad]))
            ncalls += 1
    return ncalls


# ---------------------------------------------------------------------------------------------
# Jacobi values at single points, for arrays too large for a whole oracle run
# ---------------------------------------------------------------------------------------------

def light_cone(x, prec, samples, T):
    """Value after T Jacobi steps at each sample, from the oracle on the sample's light cone.

    A value after T steps depends only on cells within distance T, so the oracle runs on the
    window of radius T + 1 around the sample with the window's outer ring held fixed (the
    array's own boundary where the window reaches it).  x is not modified."""
    n0, n1 = x.shape
    out = []
    for (i, j) in samples:
        r0, r1 = max(0, i - T - 1), min(n0, i + T + 2)
        c0, c1 = max(0, j - T - 1), min(n1, j + T + 2)
        B = x[r0:r1, c0:c1].copy()  # a copy even when the window is the whole array
        A = B.copy()
        work = np.zeros(B.shape, np.uint8)
        gi = np.arange(r0, r1)[:, None]
        gj = np.arange(c0, c1)[None, :]
        inside = (gi >= 1) & (gi < n0 - 1) & (gj >= 1) & (gj < n1 - 1)
        border = np.zeros(B.shape, bool)
        border[0, :] = border[-1, :] = border[:, 0] = border[:, -1] = True
        work[(inside & ~border)] = 1
        L = oracle.lib()
        for _ in range(T):
            rc = L.orc_jacobi2d(prec, B.shape[0], B.shape[1], B.ctypes.data, A.ctypes.data, work.ctypes.data)
            assert rc == 0
            A, B = B, A
        out.append(B[i - r0, j - c0])
    return np.array(out)


def light_cone3(x, prec, samples, T):
    """The 3-D form of light_cone (7-point stencil, orc_stencil3d)."""
    n0, n1, n2 = x.shape
    out = []
    L = oracle.lib()
    for (i, j, k) in samples:
        lo = [max(0, v - T - 1) for v in (i, j, k)]
        hi = [min(n, v + T + 2) for v, n in zip((i, j, k), (n0, n1, n2))]
        B = x[lo[0]:hi[0], lo[1]:hi[1], lo[2]:hi[2]].copy()
        A = B.copy()
        g = np.meshgrid(*[np.arange(a, b) for a, b in zip(lo, hi)], indexing="ij")
        inside = np.ones(B.shape, bool)
        for d, n in enumerate((n0, n1, n2)):
            inside &= (g[d] >= 1) & (g[d] < n - 1)
        border = np.zeros(B.shape, bool)
        for d in range(3):
            idx = [slice(None)] * 3
            idx[d] = 0
            border[tuple(idx)] = True
            idx[d] = -1
            border[tuple(idx)] = True
        work = np.ascontiguousarray((inside & ~border).astype(np.uint8))
        for _ in range(T):
            rc = L.orc_stencil3d(prec, B.shape[0], B.shape[1], B.shape[2], B.ctypes.data, A.ctypes.data,
                                 work.ctypes.data)
            assert rc == 0
            A, B = B, A
        out.append(B[i - lo[0], j - lo[1], k - lo[2]])
    return np.array(out)
