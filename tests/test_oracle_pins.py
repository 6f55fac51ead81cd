"""Pins of the CPU oracle to facts outside itself (CPU only).

Each test checks the oracle against something the paper or mathematics fixes: hand-worked
section and message sets (tests/golden/), the communication volumes printed in Table 3, closed
forms (Jacobi eigenmodes, arithmetic series), library routines for special cases (numpy's
triangular product, torch's bfloat16 rounding) and an independent version-counter simulation of
what every device must hold.
"""
import math
import os

import numpy as np
import pytest

import oracle
from oracle import Oracle, ROW, COL, BLOCK, SUM, PROD, MAX, MIN
import synthetic

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
PTYPES = {"ROW": ROW, "COL": COL, "BLOCK": BLOCK}


# ---------------------------------------------------------------------------------------------
# partitions and trapezoids
# ---------------------------------------------------------------------------------------------

def _golden_lines(name):
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                yield line


def test_partition_golden():
    n = 0
    for line in _golden_lines("partitions.txt"):
        head, boxes = line.split(":")
        t, P, lo0, hi0, lo1, hi1 = head.split()
        P = int(P)
        want = [tuple(int(v) for v in b.split()) for b in boxes.split("|")]
        got = oracle.partition_boxes(PTYPES[t], P, (int(hi0), int(hi1)),
                                     (int(lo0), int(lo1)), (int(hi0), int(hi1)))
        got = [(b[0][0], b[1][0], b[0][1], b[1][1]) for b in got]
        assert got == want, line
        n += 1
    assert n >= 8


def test_manual_partition_listing1_is_half_open():
    """Listing 1 gives device 0 rows (0,3008) and device 1 rows (3008,7232): the shared endpoint
    only makes a valid (race-free) partition with half-open bounds."""
    o = Oracle(2)
    a = o.create("a", "float", (7232, 4))
    part = o.partition_manual([((0, 0), (3008, 4)), ((3008, 0), (7232, 4))])
    o.write(a, np.zeros((7232, 4), np.float32), part)  # a definition by each device: no race
    owner, _ = a.state_get()
    assert (owner.reshape(7232, 4)[:3008] == 0).all()
    assert (owner.reshape(7232, 4)[3008:] == 1).all()


def test_trapezoid_golden():
    n = 0
    for line in _golden_lines("trapezoids.txt"):
        head, rows = line.split(":", 1)
        corners = [int(v) for v in head.split()]
        want = set()
        for item in rows.split():
            r, span = item.split(":")
            c0, c1 = span.split("-")
            for c in range(int(c0), int(c1) + 1):
                want.add((int(r), c))
        a = oracle.oracle.OArray("t", "double", (10, 10), 1)
        m = np.zeros(100, np.uint8)
        a.mask_trapezoid(corners, m)
        got = {(int(i) // 10, int(i) % 10) for i in np.nonzero(m)[0]}
        assert got == want, line
        n += 1
    assert n == 5


def test_lower_triangle_trapezoid_count():
    """Slope-1 lower triangle including the diagonal: n(n+1)/2 elements."""
    for n in (1, 2, 7, 64):
        a = oracle.oracle.OArray("t", "double", (n, n), 1)
        m = np.zeros(n * n, np.uint8)
        a.mask_trapezoid([0, 0, 0, 0, n - 1, 0, n - 1, n - 1], m)
        assert int(m.sum()) == n * (n + 1) // 2
        assert (np.tril(np.ones((n, n))) == m.reshape(n, n)).all()


# ---------------------------------------------------------------------------------------------
# hand-worked message sets (Eq. 1-4)
# ---------------------------------------------------------------------------------------------

def _run_golden_program(name):
    lines = list(_golden_lines(name))
    dims = tuple(int(v) for v in lines[0].split()[1:])
    ndev = int(lines[1].split()[1])
    o = Oracle(ndev)
    parts, arrays = {}, {}
    i = 2
    while lines[i].startswith("part"):
        _, pname, t, lo0, hi0, lo1, hi1 = lines[i].split()
        parts[pname] = o.partition(PTYPES[t], dims, (int(lo0), int(lo1)), (int(hi0), int(hi1)))
        i += 1
    checked = 0
    while i < len(lines):
        head = lines[i]
        assert head.startswith("call")
        words = head.split(":", 1)[1].split()
        i += 1
        want = {}
        while i < len(lines) and not lines[i].startswith("call"):
            if lines[i] != "none":
                lhs, rhs = lines[i].split(":", 1)
                arg = int(lhs.split()[1])
                toks = rhs.split()
                q, p = (int(v) for v in toks[0].split("->"))
                els = {tuple(int(v) for v in t.strip("()").split(",")) for t in toks[1:]}
                want.setdefault((arg, q, p), set()).update(els)
            i += 1
        names = [words[1]] if words[0] == "write" else words[3:]
        for w in names:
            if w not in arrays:
                arrays[w] = o.create(w, "double", dims)
        if words[0] == "write":
            arr = arrays[words[1]]
            o.write(arr, np.arange(arr.total, dtype=np.float64).reshape(dims), parts[words[2]])
            got = {}
        else:
            kname, part = words[1], parts[words[2]]
            args = [arrays[w] for w in words[3:]]
            msgs = o.apply(kname, part, args, scalars=(1.0, 0.0), compute=False)
            got = {}
            seen = set()
            for a_i, m in msgs.items():
                if id(args[a_i]) in seen:
                    continue
                seen.add(id(args[a_i]))
                for q in range(ndev):
                    for p in range(ndev):
                        els = m.elements(q, p)
                        if len(els):
                            got[(a_i, q, p)] = {(int(e) // dims[1], int(e) % dims[1]) for e in els}
        assert got == want, (name, head)
        checked += 1
    return checked


@pytest.mark.parametrize("name", ["messages_jacobi_p2.txt", "messages_jacobi_p3.txt",
                                  "messages_gemm_p2.txt"])
def test_message_golden(name):
    assert _run_golden_program(name) >= 5


# ---------------------------------------------------------------------------------------------
# Table 3: communication volumes printed by the paper
# ---------------------------------------------------------------------------------------------

def _table3():
    rows = {}
    for line in _golden_lines("table3_volumes.txt"):
        w = line.split()
        if w[0] == "benchmark":
            continue
        rows[w[0]] = dict(value=float(w[1]), unit=w[2], eb=int(w[3]), P=int(w[4]),
                          iters=int(w[5]), nrows=int(w[6]), rowlen=int(w[7]))
    return rows


def _to_unit(nbytes, unit):
    return nbytes / {"GiB": 2.0 ** 30, "MB": 1e6}[unit]


def test_table3_gemm_volume():
    t = _table3()["GEMM"]
    P = t["P"]
    counts = {}
    for n in (64, 96):
        o = Oracle(P)
        part = o.partition(ROW, (n, n), (0, 0), (n, n))
        A, B, C = (o.create(x, "float", (n, n)) for x in "ABC")
        for arr in (A, B, C):
            o.write(arr, None, part)
        per_call = []
        for _ in range(3):
            msgs = o.apply("gemm", part, [A, B, C], (1.0, 0.0), compute=False)
            per_call.append(sum(m.total for m in msgs.values()))
        assert per_call[1] == per_call[2] == 0  # rGDEF empty after the first all-gather
        counts[n] = per_call[0]
        assert per_call[0] == (P - 1) * n * n  # every device receives all rows it does not hold
    n = t["nrows"]
    vol = (P - 1) * n * n * t["eb"]
    assert round(_to_unit(vol, t["unit"])) == t["value"]


def _stencil_counts(kname, P, nrows, rowlen, ncalls):
    """Messages per call of the paper's Jacobi program (kernel 1 then the copy kernel) or of the
    convolution (kernel only), data partition = whole array, work = interior."""
    o = Oracle(P)
    dims = (nrows, rowlen)
    data = o.partition(ROW, dims, (0, 0), dims)
    work = o.partition(ROW, dims, (1, 1), (nrows - 1, rowlen - 1))
    B = o.create("B", "float", dims)
    A = o.create("A", "float", dims)
    o.write(B, None, data)
    o.write(A, None, data)
    per_iter = []
    for _ in range(ncalls):
        msgs = o.apply(kname, work, [B, A], compute=False)
        c = msgs[0].total
        if kname == "jacobi2d":
            c += o.apply("copy", work, [A, B], compute=False)[0].total
        per_iter.append(c)
    return per_iter


@pytest.mark.parametrize("bench", ["Jacobi", "Convolution"])
def test_table3_stencil_volume(bench):
    t = _table3()[bench]
    P, nrows = t["P"], t["nrows"]
    kname = "jacobi2d" if bench == "Jacobi" else "conv2d"
    widths = (8, 11, 17)
    per = {w: _stencil_counts(kname, P, nrows, w, 3) for w in widths}
    # messages per call are affine in the row length (whole rows, interior rows or ring cells)
    for k in range(3):
        (w0, w1, w2) = widths
        a = (per[w1][k] - per[w0][k]) / (w1 - w0)
        assert per[w2][k] == per[w0][k] + a * (w2 - w0)

    def at(k, w):
        a = (per[widths[1]][k] - per[widths[0]][k]) / (widths[1] - widths[0])
        return per[widths[0]][k] + a * (w - widths[0])

    L = t["rowlen"]
    if bench == "Jacobi":
        assert per[8][1] == per[8][2] == 2 * (P - 1) * (8 - 2)  # one interior row per face
        total = at(0, L) + (t["iters"] - 1) * at(1, L)
    else:
        assert per[8][1] == per[8][2] == 0  # no dependency across iterations
        total = at(0, L)
    assert round(_to_unit(total * t["eb"], t["unit"])) == t["value"]


# ---------------------------------------------------------------------------------------------
# values: closed forms and library special cases
# ---------------------------------------------------------------------------------------------

def _eigenmode(shape, modes):
    grids = np.meshgrid(*[np.arange(n) for n in shape], indexing="ij")
    u = np.ones(shape)
    for g, n, a in zip(grids, shape, modes):
        u = u * np.sin(math.pi * a * g / (n - 1))
    ring = np.zeros(shape, bool)
    for d in range(len(shape)):
        idx = [slice(None)] * len(shape)
        idx[d] = 0
        ring[tuple(idx)] = True
        idx[d] = shape[d] - 1
        ring[tuple(idx)] = True
    u[ring] = 0.0
    lam = sum(math.cos(math.pi * a / (n - 1)) for n, a in zip(shape, modes)) / len(shape)
    return u, lam


def _jacobi_program(shape, P, kind, values, iters, ptype=ROW, dtype="double", pingpong=False):
    o = Oracle(P)
    dims = tuple(shape)
    data = o.partition(ptype, dims, (0,) * len(dims), dims)
    work = o.partition(ptype, dims, (1,) * len(dims), tuple(n - 1 for n in dims))
    B = o.create("B", dtype, dims)
    A = o.create("A", dtype, dims)
    o.write(B, values, data)
    o.write(A, values, data)
    kname = "jacobi2d" if len(dims) == 2 else "stencil3d"
    for _ in range(iters):
        o.apply(kname, work, [B, A])
        if pingpong:
            A, B = B, A
        else:
            o.apply("copy", work, [A, B])
    return o, B, work


@pytest.mark.parametrize("shape,modes", [((17, 17), (1, 1)), ((12, 21), (2, 3)),
                                         ((9, 13), (1, 4))])
def test_jacobi_eigenmode_decay(shape, modes):
    u0, lam = _eigenmode(shape, modes)
    for it in (1, 5):
        o, B, _ = _jacobi_program(shape, 3, "jacobi2d", u0, it)
        np.testing.assert_allclose(B.G, lam ** it * u0, rtol=0, atol=1e-14)


@pytest.mark.parametrize("shape,modes", [((9, 11, 13), (1, 2, 1)), ((10, 10, 10), (3, 1, 2))])
def test_stencil3d_eigenmode_decay(shape, modes):
    u0, lam = _eigenmode(shape, modes)
    o, B, _ = _jacobi_program(shape, 4, "stencil3d", u0, 3)
    np.testing.assert_allclose(B.G, lam ** 3 * u0, rtol=0, atol=1e-14)


# The printed Jacobi step (Sec. 5) sums the four neighbours left to right: ((W + E) + N) + S with
# W = B[i][j-1], E = B[i][j+1], N = B[i-1][j], S = B[i+1][j].  With u the unit roundoff (half an
# ulp of 1), 1 + u is a tie and rounds to 1 (even), so each neighbourhood below has a result that
# follows from that order by hand; every other order of the four terms (up to swapping the first
# two, which commute) changes the bits of at least one of the three results.
#   (W, E, N, S) = (1, u, u, u):  ((1 + u) + u) + u = 1                  -> 1/4
#   (W, E, N, S) = (1, u, u, -1): ((1 + u) + u) - 1 = 0                  -> 0
#   (W, E, N, S) = (1, u, -1, u): ((1 + u) - 1) + u = u                  -> u/4
def _one_cell(dtype, dims, nbrs):
    """Run one stencil step on a 3 x 3 (x 3) array whose centre is the only work element; its
    neighbours get the values nbrs (in the kernel's operand order); returns the centre's result."""
    kname = "jacobi2d" if len(dims) == 2 else "stencil3d"
    x = np.zeros(dims, np.float64)
    c = (1,) * len(dims)
    steps = [(0, -1), (0, 1), (-1, 0), (1, 0)] if len(dims) == 2 else \
        [(0, 0, -1), (0, 0, 1), (0, -1, 0), (0, 1, 0), (-1, 0, 0), (1, 0, 0)]
    for (d, v) in zip(steps, nbrs):
        x[tuple(ci + di for ci, di in zip(c, d))] = v
    o = Oracle(1)
    B = o.create("B", dtype, dims)
    A = o.create("A", dtype, dims)
    whole = o.partition(ROW, dims, (0,) * len(dims), dims)
    work = o.partition(ROW, dims, (1,) * len(dims), (2,) * len(dims))
    o.write(B, synthetic.to_storage(x, dtype), whole)
    o.apply(kname, work, [B, A])
    return A.values64()[c]


@pytest.mark.parametrize("dtype,u", [("double", 2.0 ** -53), ("float", 2.0 ** -24), ("bf16", 2.0 ** -24)])
def test_jacobi_summation_order_as_printed(dtype, u):
    # bfloat16 storage computes in binary32, and u = 2^-24 and the results are bfloat16 numbers
    assert _one_cell(dtype, (3, 3), (1.0, u, u, u)) == 0.25
    assert _one_cell(dtype, (3, 3), (1.0, u, u, -1.0)) == 0.0
    assert _one_cell(dtype, (3, 3), (1.0, u, -1.0, u)) == u / 4


# The 3-D step sums the six face neighbours in the order x-, x+, y-, y+, z-, z+ and divides once by 6
# (correctly rounded).  With u as above:
#   (u, 1, -1, u, u, 1):    (u + 1) = 1, 1 - 1 = 0, 0 + u = u, u + u = 2u, 2u + 1 = 1 + 2u (exact)
#   (1, u, 0.5, u, -1, -1): 1 + u = 1, 1.5, 1.5 + u = 1.5 (a tie, even), 0.5, -0.5
# and every other left-to-right order of the six terms (up to swapping the first two) changes at
# least one of the two sums.
@pytest.mark.parametrize("ft,u", [(np.float64, 2.0 ** -53), (np.float32, 2.0 ** -24)])
def test_stencil3d_summation_order_as_printed(ft, u):
    dtype = "double" if ft is np.float64 else "float"
    assert _one_cell(dtype, (3, 3, 3), (u, 1.0, -1.0, u, u, 1.0)) == float(ft(1.0 + 2 * u) / ft(6.0))
    assert _one_cell(dtype, (3, 3, 3), (1.0, u, 0.5, u, -1.0, -1.0)) == float(ft(-0.5) / ft(6.0))


def _conv_program(x, w, P=3, ptype=ROW, dtype="double"):
    o = Oracle(P)
    dims = x.shape
    data = o.partition(ptype, dims, (0, 0), dims)
    work = o.partition(ptype, dims, (1, 1), (dims[0] - 1, dims[1] - 1))
    X = o.create("X", dtype, dims)
    Y = o.create("Y", dtype, dims)
    o.write(X, x, data)
    o.apply("conv2d", work, [X, Y], scalars=tuple(float(v) for v in w))
    return Y


def test_conv2d_matches_library_correlation():
    """Sec. 5's convolution in binary64 against scipy's 2-D correlation (the same weights applied
    at the same offsets, no flip) on the interior; the summation orders differ, so the bound is
    9 roundings of sum |w| |x|.  Asymmetric weights catch a transposed or flipped filter."""
    sig = pytest.importorskip("scipy.signal")
    x = synthetic.normal(23 * 31, stream=88).reshape(23, 31)
    w = synthetic.normal(9, stream=89)
    Y = _conv_program(x, w, P=4, ptype=BLOCK)
    ref = sig.correlate2d(x, w.reshape(3, 3), mode="valid")
    mag = sig.correlate2d(np.abs(x), np.abs(w.reshape(3, 3)), mode="valid")
    got = Y.G[1:-1, 1:-1]
    assert (np.abs(got - ref) <= 9 * 2.0 ** -53 * mag).all()
    assert not np.allclose(got, sig.correlate2d(x, w.reshape(3, 3).T, mode="valid"))


@pytest.mark.parametrize("dtype", ["double", "float"])
def test_conv2d_integer_exact(dtype):
    """Small integer fields and weights: every product and partial sum is an exact integer in
    both precisions, so the result equals the integer correlation exactly."""
    x = np.floor(synthetic.uniform(17 * 19, stream=90) * 200 - 100).reshape(17, 19)
    w = np.floor(synthetic.uniform(9, stream=91) * 16 - 8)
    Y = _conv_program(x.astype(np.float64 if dtype == "double" else np.float32), w, P=3, ptype=COL, dtype=dtype)
    xi, wi = x.astype(np.int64), w.astype(np.int64).reshape(3, 3)
    ref = np.zeros((15, 17), np.int64)
    for a in range(3):
        for b in range(3):
            ref += wi[a, b] * xi[a:a + 15, b:b + 17]
    assert np.array_equal(Y.G[1:-1, 1:-1].astype(np.int64), ref)


def test_conv2d_bf16_is_binary32_then_rounded():
    """bfloat16 storage: binary32 arithmetic on the decoded values, then one round to nearest even
    (torch's conversion) on the store."""
    torch = pytest.importorskip("torch")
    x = synthetic.jacobi_field((14, 16), stream=92, dtype="bf16")
    w = synthetic.normal(9, stream=93)
    yb = _conv_program(x, w, P=2, dtype="bf16").G
    x32 = oracle.bf16_to_f32(x)
    y32 = _conv_program(x32, w, P=2, dtype="float").G
    want = torch.from_numpy(y32[1:-1, 1:-1].copy()).to(torch.bfloat16).view(torch.int16).numpy().view(np.uint16)
    assert np.array_equal(yb[1:-1, 1:-1], want)


def _cov_oracle(x, P=3, correlation=False, balanced=False):
    import sys
    sys.path.insert(0, os.path.dirname(__file__))
    from cov_program import cov_prog
    from harness import OracleRun
    n, m = x.shape
    prog, _ = cov_prog(n, m, P, "double", balanced=balanced, correlation=correlation)
    orc = OracleRun(P)
    orc.run(prog, {"X": x})
    return orc.arrays


@pytest.mark.parametrize("balanced", [False, True])
def test_covariance_program_matches_numpy(balanced):
    """The oracle's covariance program (means, centring, triangular product, symmetric copy) gives
    numpy's covariance matrix; its pieces are the plain definitions: centring and the scaling are
    single IEEE operations, the copy makes C exactly symmetric."""
    x = synthetic.normal(50 * 23, stream=112).reshape(50, 23) * 3 + 1
    a = _cov_oracle(x, P=4, balanced=balanced)
    n = x.shape[0]
    assert np.allclose(a["M"].G[0], x.mean(axis=0), rtol=0, atol=1e-14 * np.abs(x).max())
    assert np.array_equal(a["Xc"].G, x - a["M"].G[0])
    C = a["C"].G
    assert np.array_equal(C, C.T)
    ref = np.cov(x, rowvar=False)
    assert np.abs(C - ref).max() <= 1e-13 * np.abs(ref).max()
    Xc = a["Xc"].G
    assert np.abs(np.triu(C) - np.triu(Xc.T @ Xc / (n - 1))).max() <= 1e-13 * np.abs(ref).max()


def test_correlation_program_matches_numpy():
    x = synthetic.normal(40 * 17, stream=113).reshape(40, 17) * np.linspace(0.5, 4, 17) + 2
    a = _cov_oracle(x, P=3, correlation=True)
    S = a["S"].G[0]
    assert np.allclose(S, np.sqrt((a["Xc"].G ** 2).sum(axis=0)), rtol=1e-15, atol=0)
    assert np.array_equal(a["Xs"].G, a["Xc"].G / S)
    C = a["C"].G
    assert np.array_equal(C, C.T)
    assert np.abs(C - np.corrcoef(x, rowvar=False)).max() <= 1e-14


def test_pingpong_equals_two_kernel_form():
    """Jacobi with kernel 2 (B = A) and with swapped arguments produce identical values."""
    x = synthetic.jacobi_field((20, 23), stream=99)
    _, B1, _ = _jacobi_program((20, 23), 3, "jacobi2d", x, 6)
    _, B2, _ = _jacobi_program((20, 23), 3, "jacobi2d", x, 6, pingpong=True)
    assert np.array_equal(B1.G, B2.G)


def test_gemm_one_partition_matches_numpy():
    n, m = 48, 40
    a, b = synthetic.tri_gemm_inputs(n, m, stream=3)
    c0 = synthetic.normal(n * m, stream=5).reshape(n, m)
    for alpha, beta in ((1.0, 0.0), (2.0, 0.5)):
        o = Oracle(1)
        part = o.partition(ROW, (n, m), (0, 0), (n, m))
        A = o.create("A", "double", (n, n))
        B = o.create("B", "double", (n, m))
        C = o.create("C", "double", (n, m))
        o.write(A, a, part if False else o.partition(ROW, (n, n), (0, 0), (n, n)))
        o.write(B, b, o.partition(ROW, (n, m), (0, 0), (n, m)))
        o.write(C, c0, part)
        o.apply("trmm", part, [A, B, C], (alpha, beta))
        ref = beta * c0 + alpha * (np.tril(a) @ b)
        u = 2.0 ** -53
        gamma = n * u / (1 - n * u)
        bound = gamma * (abs(beta * c0) + abs(alpha) * (np.abs(np.tril(a)) @ np.abs(b))) + 1e-300
        assert (np.abs(C.G - ref) <= 2 * bound).all()


def test_gemm_entries_match_full():
    n, m = 32, 24
    a, b = synthetic.tri_gemm_inputs(n, m, stream=4)
    ij = [(0, 0), (5, 7), (31, 23), (17, 0)]
    got = oracle.gemm_entries(a, b, None, 1.0, 0.0, ij)
    ref = np.tril(a) @ b
    for (i, j), g in zip(ij, got):
        assert abs(g - ref[i, j]) <= 1e-12 * (np.abs(a[i]) @ np.abs(b[:, j]))


def test_reduce_closed_forms():
    n0, n1 = 37, 29
    vals = np.arange(1, n0 * n1 + 1, dtype=np.float64).reshape(n0, n1)
    o = Oracle(4)
    part = o.partition(BLOCK, (n0, n1), (0, 0), (n0, n1))
    X = o.create("X", "double", (n0, n1))
    o.write(X, vals, part)
    N = n0 * n1
    assert o.reduce(X, SUM, part)[0] == N * (N + 1) / 2
    assert o.reduce(X, MAX, part)[0] == N
    assert o.reduce(X, MIN, part)[0] == 1
    p2 = np.full((n0, n1), 1.0)
    p2[3, 4] = 2.0 ** 10
    p2[7, 1] = 2.0 ** -3
    p2[0, 0] = 4.0
    Y = o.create("Y", "double", (n0, n1))
    o.write(Y, p2, part)
    assert o.reduce(Y, PROD, part)[0] == 2.0 ** 9
    # reduce over the interior only
    inner = o.partition(ROW, (n0, n1), (1, 1), (n0 - 1, n1 - 1))
    s, _ = o.reduce(X, SUM, inner)
    assert s == vals[1:-1, 1:-1].sum()  # small integers: exact in any order


@pytest.mark.parametrize("dtype", ["double", "float"])
def test_sqdiff_residual_integer_field(dtype):
    """The residual kernel (Sec. 5's convergence test, (X - Y)^2 into a binary64 array) on integer
    fields X[i][j] = 3i, Y[i][j] = j over a work region away from the border: every value is the
    exact integer (3i - j)^2 inside the region and 0 outside it.  (X - Y)^2 does not see the
    operand order, so the fields pin the indexing: 3i - j changes under a transposed or shifted
    index, and the region's edges under a wrong clip."""
    n0, n1 = 23, 31
    i, j = np.meshgrid(np.arange(n0), np.arange(n1), indexing="ij")
    x, y = (3 * i).astype(np.float64), j.astype(np.float64)
    o = Oracle(3)
    full = o.partition(ROW, (n0, n1), (0, 0), (n0, n1))
    work = o.partition(ROW, (n0, n1), (2, 3), (n0 - 1, n1 - 4))
    X = o.create("X", dtype, (n0, n1))
    Y = o.create("Y", dtype, (n0, n1))
    R = o.create("R", "double", (n0, n1))
    o.write(X, x.astype(np.float64 if dtype == "double" else np.float32), full)
    o.write(Y, y.astype(np.float64 if dtype == "double" else np.float32), full)
    o.apply("sqdiff", work, [X, Y, R], compute=True)
    want = np.zeros((n0, n1))
    want[2:n0 - 1, 3:n1 - 4] = ((3 * i - j) ** 2)[2:n0 - 1, 3:n1 - 4]
    assert np.array_equal(R.G.reshape(n0, n1), want)
    s, _ = o.reduce(R, SUM, work)
    assert s == float(((3 * i - j) ** 2)[2:n0 - 1, 3:n1 - 4].sum())


def test_bf16_rounding_matches_torch():
    torch = pytest.importorskip("torch")
    x = np.concatenate([
        synthetic.normal(5000, stream=11).astype(np.float32),
        np.array([0.0, -0.0, 1.0, 1.00390625, 1.005859375, 1.0029296875, 3.0e38, -3.0e38,
                  1e-40, -1e-41, np.inf, -np.inf], np.float32),
    ])
    # exact ties: lower 16 bits 0x8000 with even and odd upper halves
    ties = np.array([0x3f808000, 0x3f818000, 0xbf808000, 0x00008000, 0x7f7f8000], np.uint32).view(np.float32)
    x = np.concatenate([x, ties])
    got = oracle.f32_to_bf16(x)
    want = torch.from_numpy(x).to(torch.bfloat16).view(torch.int16).numpy().view(np.uint16)
    assert np.array_equal(got, want)
    back = oracle.bf16_to_f32(got)
    assert np.array_equal(back, torch.from_numpy(want.view(np.int16)).view(torch.bfloat16).float().numpy())


def test_jacobi_precisions_consistent():
    """binary32 and bfloat16 storage runs stay within their rounding bounds of binary64."""
    shape = (33, 40)
    x64 = synthetic.jacobi_field(shape, stream=7)
    iters = 10
    _, B64, _ = _jacobi_program(shape, 2, "jacobi2d", x64, iters)
    _, B32, _ = _jacobi_program(shape, 2, "jacobi2d", synthetic.to_storage(x64, "float"), iters,
                                dtype="float")
    _, Bbf, _ = _jacobi_program(shape, 2, "jacobi2d", synthetic.to_storage(x64, "bf16"), iters,
                                dtype="bf16")
    ref = B64.G
    scale = np.abs(ref).max()
    err32 = np.abs(B32.G.astype(np.float64) - ref).max() / scale
    errbf = np.abs(oracle.bf16_to_f32(Bbf.G).astype(np.float64) - ref).max() / scale
    assert err32 <= 3 * (iters + 1) * 2.0 ** -24
    assert errbf <= 3 * (iters + 1) * 2.0 ** -8
    assert err32 > 0 and errbf > err32


# ---------------------------------------------------------------------------------------------
# independent simulation: versioned per-device copies
# ---------------------------------------------------------------------------------------------

class VersionSim:
    """Every definition bumps an element's version; every device keeps the version of its copy.
    A correct message set makes every used element current, sends only stale elements, and
    sends from the device that made the current version (the last writer)."""

    def __init__(self, P, total):
        self.ver = np.zeros(total, np.int64)
        self.writer = np.full(total, -1)
        self.copy = np.zeros((P, total), np.int64)

    def check_use(self, use, msgs):
        P = self.copy.shape[0]
        for p in range(P):
            sent = msgs.src[p] >= 0
            assert not (sent & ~use[p].astype(bool)).any()          # only used elements move
            assert (self.copy[p][sent] < self.ver[sent]).all()      # only stale elements move
            q = msgs.src[p][sent]
            assert (q == self.writer[sent]).all()                   # from the last writer
            assert (q != p).all()
            assert (self.copy[q, np.nonzero(sent)[0]] == self.ver[sent]).all()
            self.copy[p][sent] = self.ver[sent]
            u = use[p].astype(bool)
            assert (self.copy[p][u] == self.ver[u]).all()           # every use sees the latest

    def define(self, dmask):
        for p in range(self.copy.shape[0]):
            d = dmask[p].astype(bool)
            self.ver[d] += 1
            self.writer[d] = p
            self.copy[p][d] = self.ver[d]


@pytest.mark.parametrize("seed", range(6))
def test_messages_against_version_simulation(seed):
    rng = synthetic.Rng(stream=1000 + seed)
    n0, n1 = rng.randint(6, 14), rng.randint(6, 14)
    P = rng.randint(2, 5)
    dims = (n0, n1)
    o = Oracle(P)
    X = o.create("X", "double", dims)
    sim = VersionSim(P, X.total)
    parts = []
    for _ in range(3):
        t = [ROW, COL, BLOCK][rng.randint(0, 2)]
        lo = (rng.randint(0, 2), rng.randint(0, 2))
        hi = (n0 - rng.randint(0, 2), n1 - rng.randint(0, 2))
        parts.append(o.partition(t, dims, lo, hi))
    for step in range(12):
        part = parts[rng.randint(0, len(parts) - 1)]
        kind = rng.randint(0, 2)
        if kind == 0:  # a use by offsets (in-place jacobi-like use, defs elsewhere)
            offs = [(rng.randint(-2, 2), rng.randint(-2, 2)) for _ in range(rng.randint(1, 4))]
            if rng.uniform() < 0.3:
                offs.append((0, oracle.ALL))
            use = o._clause_masks(X, part, offs, None)
            msgs = o._use(X, use)
            sim.check_use(use, msgs)
        elif kind == 1:  # a definition of the partition's work boxes
            d = o._region_masks(X, part)
            o._def(X, d)
            sim.define(d)
        else:  # absolute boxes and trapezoids: use then define
            use = np.zeros((P, X.total), np.uint8)
            for p in range(P):
                r0, r1 = sorted((rng.randint(0, n0 - 1), rng.randint(0, n0 - 1)))
                X.mask_trapezoid([r0, 0, r0, rng.randint(0, n1 - 1), r1, 0, r1, n1 - 1], use[p])
            msgs = o._use(X, use)
            sim.check_use(use, msgs)
        # GDEF bookkeeping agrees with the simulation: sGDEF_{p,q} = written by p, stale on q
        owner, have = X.state_get()
        assert ((owner >= 0) == (sim.writer >= 0)).all()
        assert (owner == sim.writer).all()
        for p in range(P):
            assert ((have[p] == 1) == (sim.copy[p] == sim.ver)).all()
        q0 = rng.randint(0, P - 1)
        p0 = (q0 + 1) % P
        sg = X.sgdef(q0, p0).astype(bool)
        assert (sg == ((sim.writer == q0) & (sim.copy[p0] < sim.ver))).all()


def test_send_recv_symmetry_and_exactly_once():
    """RECV_{p,q} (Eq. 2) is SEND_{q,p} (Eq. 1) and each used element arrives at most once."""
    o, B, work = _jacobi_program((16, 18), 4, "jacobi2d",
                                 synthetic.jacobi_field((16, 18), stream=1), 0, ptype=BLOCK)
    A = o.create("A2", "double", (16, 18))
    msgs = o.apply("jacobi2d", work, [B, A])
    m = msgs[0]
    for p in range(4):
        srcs = m.src[p]
        assert ((srcs == -1) | ((srcs >= 0) & (srcs != p))).all()
        # counts[q, p] agree with the element lists
        for q in range(4):
            assert m.counts[q, p] == (srcs == q).sum()


def test_race_detected():
    o = Oracle(2)
    X = o.create("X", "double", (4, 4))
    part = o.partition_manual([((0, 0), (3, 4)), ((2, 0), (4, 4))])  # rows 2 overlap
    with pytest.raises(ValueError):
        o.write(X, np.zeros((4, 4)), part)


def test_sampled_mode_agrees_with_full_mode():
    dims = (30, 26)
    P = 6
    coords = [(i, j) for i in range(dims[0]) for j in range(dims[1]) if (i * 7 + j * 3) % 5 == 0]
    flat = [i * dims[1] + j for i, j in coords]
    res = []
    for c in (None, coords):
        o = Oracle(P)
        data = o.partition(BLOCK, dims, (0, 0), dims)
        work = o.partition(BLOCK, dims, (1, 1), (dims[0] - 1, dims[1] - 1))
        B = o.create("B", "double", dims, coords=c)
        A = o.create("A", "double", dims, coords=c)
        o.write(B, None, data)
        o.write(A, None, data)
        out = []
        for _ in range(3):
            out.append(o.apply("jacobi2d", work, [B, A], compute=False)[0].src.copy())
            A, B = B, A
        res.append(out)
    for full, samp in zip(*res):
        assert np.array_equal(full[:, flat], samp)


def test_offsets_golden():
    n = 0
    for line in _golden_lines("offsets.txt"):
        work, offs, rows = (x.strip() for x in line.split("|"))
        lo0, hi0, lo1, hi1 = (int(v) for v in work.split())
        offsets = []
        for tok in offs.split():
            offsets.append(tuple(oracle.ALL if v == "*" else int(v) for v in tok.split(",")))
        want = set()
        for item in rows.split():
            r, span = item.split(":")
            c0, c1 = span.split("-")
            want |= {(int(r), c) for c in range(int(c0), int(c1) + 1)}
        a = oracle.oracle.OArray("t", "double", (6, 8), 1)
        m = np.zeros(48, np.uint8)
        a.mask_offsets((lo0, lo1), (hi0, hi1), offsets, m)
        assert {(int(i) // 8, int(i) % 8) for i in np.nonzero(m)[0]} == want, line
        n += 1
    assert n == 6
