"""Seeded synthetic inputs shaped like the paper's workloads.

This module only draws numbers and shapes.  It holds none of the method's arithmetic (no
sections, no messages, no stencils) and is the one module that both the oracle-side tests and the
GPU-side tests import.

Generator: splitmix64 (Steele, Lea & Flood, "Fast splittable pseudorandom number generators",
OOPSLA 2014), counter based: output i of stream s under seed S is mix(base + (i + 1) * GAMMA) with
base = mix(S + (s + 1) * GAMMA).  Uniforms are (x >> 11) * 2^-53 in [0, 1); normals come from the
Box-Muller transform of two uniforms.  Master seed 1809; the stream is the workload number.

Workload recipes (the paper's PolyBench/ACC inputs are not available; these stand in with the
same shapes):
  * Jacobi 2-D: uniform[0,1) field, the outermost ring (the Dirichlet boundary) set to 0.
  * 3-D 7-point: the same in 3-D, plus 37 boxes tiling the cube with extents 16..256 (k-d cuts).
  * triangular GEMM: A with N(0,1) on and below the diagonal and 0 above; B with N(0,1).
  * batch of Jacobi instances: side lengths log-uniform in [64, 2048], 2..16 row or column parts.
"""
import math

import numpy as np

MASTER_SEED = 1809
GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def _mix(z):
    z = np.asarray(z, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def u64(n, stream, seed=MASTER_SEED, offset=0):
    """n raw 64-bit outputs of (seed, stream), starting at output number `offset`."""
    with np.errstate(over="ignore"):
        base = _mix(np.uint64(seed) + np.uint64(stream + 1) * GAMMA)
        i = np.arange(offset + 1, offset + n + 1, dtype=np.uint64)
        return _mix(base + i * GAMMA)


def uniform(n, stream, seed=MASTER_SEED, offset=0):
    """n doubles in [0, 1)."""
    x = u64(n, stream, seed, offset)
    return (x >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def normal(n, stream, seed=MASTER_SEED, offset=0):
    """n standard normal doubles (Box-Muller on consecutive uniform pairs)."""
    m = (n + 1) // 2
    u = uniform(2 * m, stream, seed, 2 * offset)
    u1 = 1.0 - u[0::2]  # (0, 1]
    u2 = u[1::2]
    r = np.sqrt(-2.0 * np.log(u1))
    z = np.empty(2 * m)
    z[0::2] = r * np.cos(2.0 * math.pi * u2)
    z[1::2] = r * np.sin(2.0 * math.pi * u2)
    return z[:n]


class Rng:
    """Sequential draws from one stream (for shapes and choices)."""

    def __init__(self, stream, seed=MASTER_SEED):
        self.stream = stream
        self.seed = seed
        self.pos = 0

    def uniform(self):
        v = uniform(1, self.stream, self.seed, self.pos)[0]
        self.pos += 1
        return float(v)

    def randint(self, lo, hi):
        """Uniform integer in [lo, hi] inclusive."""
        return lo + min(int(self.uniform() * (hi - lo + 1)), hi - lo)


def to_storage(x64, dtype):
    """Round binary64 values to the storage type: 'double', 'float' or 'bf16' (bit pattern,
    uint16, round to nearest even via torch's CPU conversion)."""
    if dtype == "double":
        return np.ascontiguousarray(x64, dtype=np.float64)
    if dtype == "float":
        return np.ascontiguousarray(x64, dtype=np.float32)
    if dtype == "bf16":
        import torch
        t = torch.from_numpy(np.ascontiguousarray(x64, dtype=np.float32)).to(torch.bfloat16)
        return t.view(torch.int16).numpy().view(np.uint16).copy()
    raise ValueError(dtype)


def jacobi_field(shape, stream, dtype="double", seed=MASTER_SEED):
    """uniform[0,1) field with the outermost ring set to 0 (zero Dirichlet boundary)."""
    n = int(np.prod(shape))
    x = uniform(n, stream, seed).reshape(shape)
    ring = np.zeros(shape, bool)
    for d in range(len(shape)):
        idx = [slice(None)] * len(shape)
        idx[d] = 0
        ring[tuple(idx)] = True
        idx[d] = shape[d] - 1
        ring[tuple(idx)] = True
    x[ring] = 0.0
    return to_storage(x, dtype)


def tri_gemm_inputs(n, m, stream, dtype="double", seed=MASTER_SEED):
    """A (n x n) with N(0,1) on and below the diagonal, 0 above; B (n x m) with N(0,1)."""
    a = normal(n * n, stream, seed).reshape(n, n)
    a = np.tril(a)
    b = normal(n * m, stream, seed, offset=(n * n + 1) // 2).reshape(n, m)
    return to_storage(a, dtype), to_storage(b, dtype)


def kd_boxes(n, nboxes, stream, min_ext=16, max_ext=256, seed=MASTER_SEED, max_tries=64):
    """Boxes tiling [0, n)^3 with every extent in [min_ext, max_ext], from seeded cuts.

    1. While a box has an extent > max_ext, cut its largest such dimension at a uniform position
       in [min_ext, ext - min_ext].
    2. Then, until there are `nboxes` boxes, pick a uniform box among those with some extent
       >= 2 * min_ext, a uniform such dimension, and cut it uniformly in [min_ext, ext - min_ext].
    Returns a list of (lo, hi) triples.  Reseeds (next seed) when nboxes is unreachable.
    """
    for attempt in range(max_tries):
        rng = Rng(stream, seed + attempt)
        boxes = [((0, 0, 0), (n, n, n))]
        ok = True
        while True:
            big = [i for i, (lo, hi) in enumerate(boxes)
                   if max(hi[d] - lo[d] for d in range(3)) > max_ext]
            if not big:
                break
            i = big[0]
            lo, hi = boxes[i]
            ext = [hi[d] - lo[d] for d in range(3)]
            d = max(range(3), key=lambda k: ext[k])
            cut = lo[d] + rng.randint(min_ext, ext[d] - min_ext)
            boxes[i:i + 1] = _cut(lo, hi, d, cut)
        if len(boxes) > nboxes:
            ok = False
        while ok and len(boxes) < nboxes:
            cand = [i for i, (lo, hi) in enumerate(boxes)
                    if max(hi[d] - lo[d] for d in range(3)) >= 2 * min_ext]
            if not cand:
                ok = False
                break
            i = cand[rng.randint(0, len(cand) - 1)]
            lo, hi = boxes[i]
            dims = [d for d in range(3) if hi[d] - lo[d] >= 2 * min_ext]
            d = dims[rng.randint(0, len(dims) - 1)]
            cut = lo[d] + rng.randint(min_ext, hi[d] - lo[d] - min_ext)
            boxes[i:i + 1] = _cut(lo, hi, d, cut)
        if ok and len(boxes) == nboxes:
            return boxes
    raise RuntimeError("kd_boxes: no tiling with %d boxes" % nboxes)


def _cut(lo, hi, d, cut):
    hi1 = list(hi)
    hi1[d] = cut
    lo2 = list(lo)
    lo2[d] = cut
    return [(tuple(lo), tuple(hi1)), (tuple(lo2), tuple(hi))]


def jacobi_instances(count, stream, lo=64, hi=2048, pmin=2, pmax=16, seed=MASTER_SEED):
    """Independent Jacobi instances: (rows, cols, nparts, 'ROW'|'COL') per instance.
    rows and cols independently round(lo * (hi/lo)^u), u ~ U[0,1); nparts ~ U{pmin..pmax};
    ROW or COL with probability 1/2.  The part count is capped so every part has work."""
    rng = Rng(stream, seed)
    out = []
    ratio = hi / lo
    for _ in range(count):
        r = int(round(lo * ratio ** rng.uniform()))
        c = int(round(lo * ratio ** rng.uniform()))
        P = rng.randint(pmin, pmax)
        kind = "ROW" if rng.uniform() < 0.5 else "COL"
        split = (r if kind == "ROW" else c) - 2
        P = max(1, min(P, split))
        out.append((r, c, P, kind))
    return out
