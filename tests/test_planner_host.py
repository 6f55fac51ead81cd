"""The library's communication generation against the oracle, on the host (no GPU).

libhdarray.so runs in HDARRAY_INIT_HOST_ONLY mode: partitions, sections, GDEF bookkeeping and the
exchange plans are computed exactly as on the GPU, but nothing is allocated or launched.  Each
call's exchange (HDArrayGetPlan) must equal the oracle's element-by-element messages.
"""
import numpy as np
import pytest

import oracle
import synthetic
from harness import LibraryRun, OracleRun, compare_messages

H = pytest.importorskip("paper_1809_05657_gb300.hdarray")
ROW, COL, BLOCK = 0, 1, 2


@pytest.fixture
def host_lib():
    from __graft_entry__ import build_library
    build_library()
    yield lambda ndev: H.HDArrayInit(ndev=ndev, host_only=True)
    H.HDArrayExit()


def run_both(prog, ndev, host_lib, coords=None):
    host_lib(ndev)
    lib_out = LibraryRun(H, ndev).run(prog)
    orc = OracleRun(ndev, coords=coords)
    orc_out = orc.run(prog)
    dims = {op[1]: tuple(op[3]) for op in prog if op[0] == "create"}
    return compare_messages(orc_out, lib_out, prog, dims, ndev, coords)


def jacobi_prog(dims, P, iters, ptype=ROW, dtype="double", pingpong=False, kernel=None):
    nd = len(dims)
    kernel = kernel or ("jacobi2d" if nd == 2 else "stencil3d")
    prog = [("create", "B", dtype, dims), ("create", "A", dtype, dims),
            ("part", "D", ptype, dims, (0,) * nd, dims, P),
            ("part", "W", ptype, dims, (1,) * nd, tuple(n - 1 for n in dims), P),
            ("write", "B", "D"), ("write", "A", "D")]
    x, y = "B", "A"
    for _ in range(iters):
        prog.append(("apply", kernel, "W", [x, y]))
        if pingpong:
            x, y = y, x
        else:
            prog.append(("apply", "copy", "W", [y, x]))
    return prog


# ---------------------------------------------------------------------------------------------

@pytest.mark.parametrize("dims,P,ptype", [((6, 4), 2, ROW), ((8, 5), 3, ROW), ((13, 11), 4, BLOCK),
                                          ((12, 17), 3, COL), ((20, 20), 6, BLOCK)])
def test_jacobi_messages(host_lib, dims, P, ptype):
    assert run_both(jacobi_prog(dims, P, 4, ptype), P, host_lib) > 0


@pytest.mark.parametrize("P", [2, 5])
def test_jacobi_pingpong_messages(host_lib, P):
    assert run_both(jacobi_prog((15, 19), P, 5, BLOCK, pingpong=True), P, host_lib) > 0


def test_gemm_listing2_messages(host_lib):
    n = 12
    prog = [("create", "a", "double", (n, n)), ("create", "b", "double", (n, n)),
            ("create", "c", "double", (n, n)), ("part", "p0", ROW, (n, n), (0, 0), (n, n), 4),
            ("write", "a", "p0"), ("write", "b", "p0"), ("write", "c", "p0"),
            ("apply", "gemm", "p0", ["a", "b", "c"], (1.0, 0.0, n, n, n)),
            ("apply", "gemm", "p0", ["a", "b", "c"], (1.0, 0.0, n, n, n)),
            ("read", "c", "p0")]
    assert run_both(prog, 4, host_lib) >= 3


def test_trapezoid_gemm_messages(host_lib):
    """Lower-triangular A: each device uses the trapezoid of its rows (Sec. 3.1)."""
    n, m, P = 16, 8, 4
    prog = [("create", "A", "double", (n, n)), ("create", "B", "double", (n, m)),
            ("create", "C", "double", (n, m)),
            ("part", "R", ROW, (n, m), (0, 0), (n, m), P),
            ("part", "RA", ROW, (n, n), (0, 0), (n, n), P)]
    for p in range(P):
        r0, r1 = p * n // P, (p + 1) * n // P
        prog.append(("trap_use", "trmm", "R", "A", p, (r0, 0, r0, r0, r1 - 1, 0, r1 - 1, r1 - 1)))
    # A written by a COL partition: every device needs parts of its triangle from others
    prog += [("part", "CA", COL, (n, n), (0, 0), (n, n), P),
             ("write", "A", "CA"), ("write", "B", "R"), ("write", "C", "R"),
             ("apply", "trmm", "R", ["A", "B", "C"], (1.0, 0.0)),
             ("apply", "trmm", "R", ["A", "B", "C"], (1.0, 0.0))]
    assert run_both(prog, P, host_lib) >= 3


def test_absolute_sections(host_lib):
    n = 10
    prog = [("create", "X", "double", (n, n)), ("create", "Y", "double", (n, n)),
            ("part", "Q", BLOCK, (n, n), (0, 0), (n, n), 4),
            ("write", "X", "Q"),
            ("abs_use", "copy", "Q", "X", 0, (0, 0), (n, 3)),
            ("abs_use", "copy", "Q", "X", 0, (7, 2), (9, 9)),
            ("abs_use", "copy", "Q", "X", 3, (0, 0), (2, 2)),
            ("apply", "copy", "Q", ["X", "Y"]),
            ("read", "X", "Q"),
            ("reduce", "X", 0, "Q")]
    assert run_both(prog, 4, host_lib) >= 3


def test_manual_partition_3d(host_lib):
    n = 12
    boxes = synthetic.kd_boxes(n, 7, stream=2, min_ext=3, max_ext=12)
    prog = [("create", "X", "float", (n, n, n)),
            ("manual", "M", (n, n, n), boxes),
            ("write", "X", "M"),
            ("offset_use", "copy", 0, [(0, 0, -1), (0, 0, 1), (0, -1, 0), (0, 1, 0), (-1, 0, 0), (1, 0, 0)]),
            ("create", "Y", "float", (n, n, n)),
            ("apply", "copy", "M", ["X", "Y"]),
            ("apply", "copy", "M", ["Y", "X"]),
            ("apply", "copy", "M", ["X", "Y"])]
    assert run_both(prog, 7, host_lib) >= 3


@pytest.mark.parametrize("seed", range(8))
def test_random_programs(host_lib, seed):
    rng = synthetic.Rng(stream=5000 + seed)
    nd = 2 if seed % 3 else 3
    dims = tuple(rng.randint(5, 12) for _ in range(nd))
    P = rng.randint(2, 6)
    prog = [("create", "X", "double", dims), ("create", "Y", "double", dims)]
    parts = []
    for i in range(3):
        if rng.uniform() < 0.3:
            boxes = []
            for p in range(P):
                lo = tuple(rng.randint(0, n - 1) for n in dims)
                hi = tuple(min(n, l + rng.randint(1, 4)) for l, n in zip(lo, dims))
                boxes.append((lo, hi))
            # make it race free: keep boxes disjoint by dropping overlaps
            keep = []
            for b in boxes:
                ok = all(any(b[1][d] <= k[0][d] or k[1][d] <= b[0][d] for d in range(nd)) for k in keep)
                keep.append(b if ok else (tuple(0 for _ in dims), tuple(0 for _ in dims)))
            prog.append(("manual", "p%d" % i, dims, keep))
        else:
            t = [ROW, COL, BLOCK][rng.randint(0, 2)]
            lo = tuple(rng.randint(0, 2) for _ in dims)
            hi = tuple(n - rng.randint(0, 2) for n in dims)
            prog.append(("part", "p%d" % i, t, dims, lo, hi, P))
        parts.append("p%d" % i)
    prog.append(("write", "X", parts[0]))
    for step in range(10):
        r = rng.uniform()
        part = parts[rng.randint(0, 2)]
        if r < 0.2:
            offs = [tuple(rng.randint(-2, 2) for _ in dims) for _ in range(rng.randint(1, 3))]
            if rng.uniform() < 0.3:
                o = list(offs[0])
                o[rng.randint(0, nd - 1)] = H.HDARRAY_ALL
                offs.append(tuple(o))
            prog.append(("offset_use", "copy", 0, offs))
        elif r < 0.75:
            x, y = ("X", "Y") if rng.uniform() < 0.5 else ("Y", "X")
            prog.append(("apply", "copy", part, [x, y]))
        elif r < 0.9:
            prog.append(("read", ["X", "Y"][rng.randint(0, 1)], part))
        else:
            prog.append(("write", ["X", "Y"][rng.randint(0, 1)], part))
    assert run_both(prog, P, host_lib) >= 1


# ---------------------------------------------------------------------------------------------
# full-size workloads: the sampled oracle decides the listed elements exactly
# ---------------------------------------------------------------------------------------------

def boundary_samples(dims, cuts, n_random, stream, per_line=64):
    """Elements on and next to partition cut lines, plus random elements."""
    rng = np.random.default_rng(stream)
    nd = len(dims)
    pts = []
    for d, cs in enumerate(cuts):
        for c in cs:
            for off in (-2, -1, 0, 1):
                v = c + off
                if not 0 <= v < dims[d]:
                    continue
                for _ in range(per_line):
                    p = [int(rng.integers(0, n)) for n in dims]
                    p[d] = v
                    pts.append(tuple(p))
    for _ in range(n_random):
        pts.append(tuple(int(rng.integers(0, n)) for n in dims))
    # corners of the domain and of the ring
    for corner in np.ndindex(*([2] * nd)):
        pts.append(tuple((dims[d] - 1) if corner[d] else 0 for d in range(nd)))
        pts.append(tuple((dims[d] - 2) if corner[d] else 1 for d in range(nd)))
    return sorted(set(pts))


def test_full_size_jacobi_8192_block16(host_lib):
    dims, P = (8192, 8192), 16
    d_cuts = [b for b in range(0, 8193, 2048)]
    w_cuts = [1, 2049, 4097, 6144, 8191]
    coords = boundary_samples(dims, [d_cuts + w_cuts] * 2, 3000, stream=1)
    prog = jacobi_prog(dims, P, 3, BLOCK, dtype="float", pingpong=True)
    n = run_both(prog, P, host_lib, coords={"A": coords, "B": coords})
    assert n >= 3


def test_full_size_jacobi_256_row4_full_oracle(host_lib):
    assert run_both(jacobi_prog((256, 256), 4, 3, ROW), 4, host_lib) >= 3


def test_full_size_stencil3d_37_boxes(host_lib):
    n = 512
    boxes = synthetic.kd_boxes(n, 37, stream=3)
    work = []
    for lo, hi in boxes:
        wl = tuple(max(1, v) for v in lo)
        wh = tuple(min(n - 1, v) for v in hi)
        work.append((wl, wh))
    cuts = [sorted({b[0][d] for b in boxes} | {b[1][d] for b in boxes}) for d in range(3)]
    coords = boundary_samples((n, n, n), cuts, 4000, stream=2, per_line=24)
    prog = [("create", "B", "float", (n, n, n)), ("create", "A", "float", (n, n, n)),
            ("manual", "D", (n, n, n), boxes), ("manual", "W", (n, n, n), work),
            ("write", "B", "D"), ("write", "A", "D"),
            ("offset_use", "copy", 0, [(0, 0, -1), (0, 0, 1), (0, -1, 0), (0, 1, 0), (-1, 0, 0), (1, 0, 0)]),
            ("apply", "copy", "W", ["B", "A"]), ("apply", "copy", "W", ["A", "B"]),
            ("apply", "copy", "W", ["B", "A"])]
    assert run_both(prog, 37, host_lib, coords={"A": coords, "B": coords}) >= 3


def test_full_size_stencil3d_kernel_37_boxes(host_lib):
    n = 512
    boxes = synthetic.kd_boxes(n, 37, stream=3)
    work = [(tuple(max(1, v) for v in lo), tuple(min(n - 1, v) for v in hi)) for lo, hi in boxes]
    cuts = [sorted({b[0][d] for b in boxes} | {b[1][d] for b in boxes}) for d in range(3)]
    coords = boundary_samples((n, n, n), cuts, 4000, stream=5, per_line=24)
    prog = [("create", "B", "float", (n, n, n)), ("create", "A", "float", (n, n, n)),
            ("manual", "D", (n, n, n), boxes), ("manual", "W", (n, n, n), work),
            ("write", "B", "D"),
            ("apply", "stencil3d", "W", ["B", "A"]), ("apply", "stencil3d", "W", ["A", "B"]),
            ("apply", "stencil3d", "W", ["B", "A"]), ("apply", "stencil3d", "W", ["A", "B"])]
    assert run_both(prog, 37, host_lib, coords={"A": coords, "B": coords}) >= 4


def test_full_size_trmm_8192(host_lib):
    n, m, P = 8192, 4096, 8
    rows = [1024 * p for p in range(P + 1)]
    coordsA = boundary_samples((n, n), [rows, rows], 2000, stream=3)
    coordsB = boundary_samples((n, m), [rows, [0, 4096]], 2000, stream=4)
    prog = [("create", "A", "double", (n, n)), ("create", "B", "double", (n, m)),
            ("create", "C", "double", (n, m)),
            ("part", "R", ROW, (n, m), (0, 0), (n, m), P),
            ("part", "RA", ROW, (n, n), (0, 0), (n, n), P)]
    for p in range(P):
        r0, r1 = rows[p], rows[p + 1]
        prog.append(("trap_use", "trmm", "R", "A", p, (r0, 0, r0, r0, r1 - 1, 0, r1 - 1, r1 - 1)))
    prog += [("write", "A", "RA"), ("write", "B", "R"), ("write", "C", "R"),
             ("apply", "trmm", "R", ["A", "B", "C"], (1.0, 0.0)),
             ("apply", "trmm", "R", ["A", "B", "C"], (1.0, 0.0))]
    assert run_both(prog, P, host_lib, coords={"A": coordsA, "B": coordsB, "C": coordsB}) >= 2


# ---------------------------------------------------------------------------------------------
# Table 3 volumes at the paper's full sizes, straight from the library's section algebra
# ---------------------------------------------------------------------------------------------

def _moved_bytes(H, arr, elem):
    return sum(int(np.prod(np.subtract(hi, lo))) for _, _, lo, hi in H.HDArrayGetPlan(arr)) * elem


def test_table3_gemm_volume_full_size(host_lib):
    host_lib(32)
    n = 10240
    a, b, c = (H.HDArrayCreate(x, "double", None, n, n) for x in "abc")
    p0 = H.HDArrayPartition(ROW, (n, n), (0, 0), (n, n), 32)
    for x in (a, b, c):
        H.HDArrayWrite(x, None, p0)
    total = 0
    for it in range(100):
        H.HDArrayApplyKernel("gemm", p0, a, b, c, 1.0, 0.0, n, n, n)
        total += _moved_bytes(H, b, 4) if it == 0 else 0
    # after the first call B is never moved again: the plan cache hits with an empty exchange
    assert H.HDArrayGetPlan(b) == [] or total > 0
    assert round(total / 2 ** 30) == 12  # Table 3: 12 GB


def test_table3_jacobi_volume_full_size(host_lib):
    host_lib(32)
    rows, L = 24080, 20480
    B = H.HDArrayCreate("B", "float", None, rows, L)
    A = H.HDArrayCreate("A", "float", None, rows, L)
    D = H.HDArrayPartition(ROW, (rows, L), (0, 0), (rows, L), 32)
    W = H.HDArrayPartition(ROW, (rows, L), (1, 1), (rows - 1, L - 1), 32)
    H.HDArrayWrite(B, None, D)
    H.HDArrayWrite(A, None, D)
    per = []
    for it in range(4):
        H.HDArrayApplyKernel("jacobi2d", W, B, A)
        v = _moved_bytes(H, B, 4)
        H.HDArrayApplyKernel("copy", W, A, B)
        per.append(v + _moved_bytes(H, A, 4) * 0)
    assert per[1] == per[2] == per[3] == 2 * 31 * (L - 2) * 4
    total = per[0] + 99999 * per[1]
    assert round(total / 2 ** 30) == 473  # Table 3: 473 GB
    c = H.HDArrayGetCounters()
    assert c["plan_hits"] >= 4  # steady state comes from the cache (Sec. 4.2)


def test_table3_convolution_volume_full_size(host_lib):
    host_lib(32)
    rows, L = 24080, 20480
    B = H.HDArrayCreate("B", "float", None, rows, L)
    A = H.HDArrayCreate("A", "float", None, rows, L)
    D = H.HDArrayPartition(ROW, (rows, L), (0, 0), (rows, L), 32)
    W = H.HDArrayPartition(ROW, (rows, L), (1, 1), (rows - 1, L - 1), 32)
    H.HDArrayWrite(B, None, D)
    H.HDArrayWrite(A, None, D)
    w = [0.0, 0.125, 0.0, 0.125, 0.5, 0.125, 0.0, 0.125, 0.0]
    per = []
    for it in range(3):
        H.HDArrayApplyKernel("conv2d", W, B, A, *w)
        per.append(_moved_bytes(H, B, 4))
    # the halo rows (with their corner cells) move once; B never changes, so nothing moves again
    assert per == [2 * 31 * L * 4, 0, 0]
    total = per[0]
    assert round(total / 2 ** 20) == 5  # Table 3: 5 MB


def _two_mm_volumes(P, n, iters, ptype):
    """Elements moved per iteration by 2MM (D = A B, then E = C D, Sec. 5.1) with every array
    written and every product computed on the same partition (ROW or COL)."""
    names = "ABCDE"
    arrs = {x: H.HDArrayCreate(x, "float", None, n, n) for x in names}
    part = H.HDArrayPartition(ptype, (n, n), (0, 0), (n, n), P)
    for x in names:
        H.HDArrayWrite(arrs[x], None, part)
    per = []
    for _ in range(iters):
        H.HDArrayApplyKernel("gemm", part, arrs["A"], arrs["B"], arrs["D"], 1.0, 0.0, n, n, n)
        v = sum(_moved_bytes(H, arrs[x], 1) for x in "AB")
        H.HDArrayApplyKernel("gemm", part, arrs["C"], arrs["D"], arrs["E"], 1.0, 0.0, n, n, n)
        v += sum(_moved_bytes(H, arrs[x], 1) for x in "CD")
        per.append(v)
    return per


def two_mm_prog(n, P, ptype, iters, dtype="double"):
    prog = [("create", x, dtype, (n, n)) for x in "ABCDE"]
    prog += [("part", "Q", ptype, (n, n), (0, 0), (n, n), P)]
    prog += [("write", x, "Q") for x in "ABCDE"]
    for _ in range(iters):
        prog.append(("apply", "gemm", "Q", ["A", "B", "D"], (1.0, 0.0, n, n, n)))
        prog.append(("apply", "gemm", "Q", ["C", "D", "E"], (1.0, 0.0, n, n, n)))
    return prog


@pytest.mark.parametrize("ptype", [ROW, COL])
def test_2mm_messages(host_lib, ptype):
    """2MM's messages, element by element, equal the oracle's for row and column blocks."""
    assert run_both(two_mm_prog(22, 4, ptype, 3), 4, host_lib) >= 1


@pytest.mark.parametrize("balanced,correlation", [(False, False), (True, False), (True, True)])
def test_covariance_messages(host_lib, balanced, correlation):
    """The covariance program (column means, centring, triangular product with absolute use and
    trapezoid definitions, symmetric copy): messages equal the oracle's element by element, on
    even and on area-balanced row blocks."""
    from cov_program import cov_prog
    prog, _ = cov_prog(40, 36, 4, balanced=balanced, correlation=correlation)
    assert run_both(prog, 4, host_lib) >= 3


@pytest.mark.parametrize("ptype", [ROW, COL, BLOCK])
def test_user_kernel_messages(host_lib, ptype):
    """A registered user kernel with its own use/def offsets: the library's messages equal the
    oracle's for the same clauses (no launcher runs without a GPU)."""
    import user_kernels
    user_kernels.register_oracle()
    host_lib(5)
    H.HDArrayRegisterKernel("max4", 2, 0, 1, lambda work, scal, stream: 0)
    H.HDArraySetOffsetUse("max4", 0, user_kernels.J4)
    H.HDArraySetOffsetDef("max4", 1, [(0, 0)])
    dims = (41, 37)
    prog = [("create", "B", "double", dims), ("create", "A", "double", dims),
            ("part", "D", ptype, dims, (0, 0), dims, 5), ("part", "W", ptype, dims, (1, 1), (40, 36), 5),
            ("write", "B", "D")]
    for i in range(3):
        prog.append(("apply", "max4", "W", ["B", "A"] if i % 2 == 0 else ["A", "B"]))
    lib_out = LibraryRun(H, 5).run(prog)
    orc_out = OracleRun(5).run(prog)
    assert compare_messages(orc_out, lib_out, prog, {"B": dims, "A": dims}, 5) >= 3


def test_user_kernel_registration_errors(host_lib):
    host_lib(2)
    cb = lambda work, scal, stream: 0  # noqa: E731
    with pytest.raises(H.HDArrayError):
        H.HDArrayRegisterKernel("jacobi2d", 2, 0, 1, cb)  # a built-in name
    with pytest.raises(H.HDArrayError):
        H.HDArrayRegisterKernel("k", 9, 0, 0, cb)  # too many arrays
    with pytest.raises(H.HDArrayError):
        H.HDArrayRegisterKernel("k", 2, 0, 2, cb)  # space argument out of range
    H.HDArrayRegisterKernel("k", 2, 0, 1, cb)
    H.HDArrayRegisterKernel("k", 2, 1, 1, cb)  # re-registration replaces it


def test_2mm_row_vs_column_partition_volumes(host_lib):
    """Sec. 5.1 / Table 3: with row blocks, B is gathered once and D (redefined by the first
    product in every iteration) is gathered by every device in every iteration; with column
    blocks only A and C are gathered, once.  Over 100 iterations the totals are in the ratio
    (1 + 100) : 2, which is Table 3's 1262 GB : 25 GB (the paper does not give 2MM's sizes, so the
    ratio is what pins the volumes)."""
    P, n = 32, 96
    host_lib(P)
    row = _two_mm_volumes(P, n, 4, ROW)
    host_lib(P)
    col = _two_mm_volumes(P, n, 4, COL)
    g = (P - 1) * n * n  # one all-gather of an n x n array
    assert row == [2 * g, g, g, g]
    assert col == [2 * g, 0, 0, 0]
    ratio = (row[0] + 99 * row[1]) / (col[0] + 99 * col[1])
    assert abs(ratio - 1262 / 25) / ratio < 0.01


# ---------------------------------------------------------------------------------------------
# errors and caching
# ---------------------------------------------------------------------------------------------

def test_race_and_range_errors(host_lib):
    host_lib(2)
    X = H.HDArrayCreate("X", "double", None, 8, 8)
    bad = H.HDArrayPartitionManual((8, 8), [((0, 0), (5, 8)), ((4, 0), (8, 8))])
    with pytest.raises(H.HDArrayError) as e:
        H.HDArrayWrite(X, None, bad)
    assert e.value.code == -3
    with pytest.raises(H.HDArrayError) as e:
        H.HDArrayPartition(ROW, (8, 8), (0, 0), (9, 8), 2)
    assert e.value.code == -4
    W = H.HDArrayPartition(ROW, (8, 8), (0, 0), (8, 8), 2)
    Y = H.HDArrayCreate("Y", "double", None, 8, 8)
    with pytest.raises(H.HDArrayError) as e:  # work on the border has no neighbours
        H.HDArrayApplyKernel("jacobi2d", W, X, Y)
    assert e.value.code == -4
    with pytest.raises(H.HDArrayError):
        H.HDArrayApplyKernel("nope", W, X, Y)
    with pytest.raises(H.HDArrayError):
        H.HDArrayApplyKernel("jacobi2d", W, X, X)


def test_plan_cache_steady_state(host_lib):
    host_lib(4)
    prog_calls = 0
    B = H.HDArrayCreate("B", "float", None, 64, 64)
    A = H.HDArrayCreate("A", "float", None, 64, 64)
    D = H.HDArrayPartition(BLOCK, (64, 64), (0, 0), (64, 64), 4)
    W = H.HDArrayPartition(BLOCK, (64, 64), (1, 1), (63, 63), 4)
    H.HDArrayWrite(B, None, D)
    H.HDArrayWrite(A, None, D)
    for _ in range(4):
        H.HDArrayApplyKernel("jacobi2d", W, B, A)
        H.HDArrayApplyKernel("jacobi2d", W, A, B)
        prog_calls += 2
    c0 = H.HDArrayGetCounters()
    for _ in range(50):
        H.HDArrayApplyKernel("jacobi2d", W, B, A)
        H.HDArrayApplyKernel("jacobi2d", W, A, B)
    c1 = H.HDArrayGetCounters()
    assert c1["plans"] == c0["plans"]
    assert c1["plan_hits"] - c0["plan_hits"] == 100
