"""A user kernel for the tests: the maximum of the four face neighbours, Y[i][j] =
max(X[i-1][j], X[i+1][j], X[i][j-1], X[i][j+1]) (exact in any precision), and Y = a X + b with two
scalars.  The device side is plain torch on views of the library's buffers (the user's code; the
exchange before it is the library's); the oracle side is numpy on the global array."""

import numpy as np

import oracle

J4 = [(0, -1), (0, 1), (-1, 0), (1, 0)]


def oracle_max4(o, arrs, work, scal):
    X, Y = arrs
    g, w = X.G, work.reshape(X.dims)
    out = np.maximum(np.maximum(g[:-2, 1:-1], g[2:, 1:-1]), np.maximum(g[1:-1, :-2], g[1:-1, 2:]))
    inner = w[1:-1, 1:-1].astype(bool)
    Y.G[1:-1, 1:-1][inner] = out[inner]


def oracle_axpb(o, arrs, work, scal):
    X, Y = arrs
    a, b = scal
    m = work.reshape(X.dims).astype(bool)
    Y.G[m] = (X.G[m] * X.G.dtype.type(a) + X.G.dtype.type(b)).astype(X.G.dtype)


def register_oracle():
    oracle.KERNELS["max4"] = oracle.KernelSpec(2, {0: J4}, {1: [(0, 0)]}, oracle_max4)
    oracle.KERNELS["axpb"] = oracle.KernelSpec(2, {0: [(0, 0)]}, {1: [(0, 0)]}, oracle_axpb, nscal=2)


class _View:
    def __init__(self, ptr, shape, strides, typestr):
        self.__cuda_array_interface__ = {"shape": shape, "strides": strides, "typestr": typestr,
                                         "data": (ptr, False), "version": 3}


def view(torch, w, arg, r0, r1, c0, c1, dtype):
    """torch view of rows [r0, r1) x columns [c0, c1) of argument `arg`'s buffer."""
    es = np.dtype(dtype).itemsize
    ptr = w.buf[arg] + ((r0 - w.buf_lo[arg][0]) * w.buf_stride[arg][0] + (c0 - w.buf_lo[arg][1])) * es
    return torch.as_tensor(_View(ptr, (r1 - r0, c1 - c0), (w.buf_stride[arg][0] * es, es), np.dtype(dtype).str),
                           device="cuda")


def max4_launcher(torch, dtype):
    def launch(work, scal, stream):
        with torch.cuda.stream(torch.cuda.ExternalStream(stream)):
            for w in work:
                r0, r1, c0, c1 = w.lo[0], w.hi[0], w.lo[1], w.hi[1]
                x = view(torch, w, 0, r0 - 1, r1 + 1, c0 - 1, c1 + 1, dtype)
                y = view(torch, w, 1, r0, r1, c0, c1, dtype)
                y.copy_(torch.maximum(torch.maximum(x[:-2, 1:-1], x[2:, 1:-1]), torch.maximum(x[1:-1, :-2], x[1:-1, 2:])))
        return 0
    return launch


def axpb_launcher(torch, dtype):
    def launch(work, scal, stream):
        a, b = scal
        with torch.cuda.stream(torch.cuda.ExternalStream(stream)):
            for w in work:
                x = view(torch, w, 0, w.lo[0], w.hi[0], w.lo[1], w.hi[1], dtype)
                y = view(torch, w, 1, w.lo[0], w.hi[0], w.lo[1], w.hi[1], dtype)
                y.copy_(x * a + b)
        return 0
    return launch
