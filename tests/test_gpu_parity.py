"""GPU parity: the CUDA path through the C ABI against the oracle.

Bar: section sets (every call's exchange) and every copied or computed element bit-exact; the
Jacobi kernels sum in the paper's order in the storage precision, so their results are bit-exact
too.  Floating-point results with a different summation order (reductions, GEMM) are within the
bounds stated in each test.
"""
import ctypes

import numpy as np
import pytest

import oracle
import synthetic
from harness import LibraryRun, OracleRun, compare_messages, light_cone, light_cone3

pytestmark = pytest.mark.gpu

H = pytest.importorskip("paper_1809_05657_gb300.hdarray")
ROW, COL, BLOCK = 0, 1, 2
NP = {"double": np.float64, "float": np.float32, "bf16": np.uint16}


@pytest.fixture
def gpu_lib():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from __graft_entry__ import build_library
    build_library()
    torch.cuda.init()
    yield lambda ndev: H.HDArrayInit(ndev=ndev)
    H.HDArrayExit()


def device_buffers_match(lib_run, orc_run, names):
    """Every element a device holds as current equals the global value, bit for bit."""
    for name in names:
        a = lib_run.arrays[name]
        oa = orc_run.arrays[name]
        owner, have = oa.state_get()
        dims = oa.dims
        n3 = list(dims) + [1] * (3 - len(dims))
        for p in range(oa.P):
            ptr, lo, hi, st = H.HDArrayGetDeviceBuffer(a, p)
            if ptr is None:
                assert not have[p].any() or (owner[have[p].astype(bool)] == -1).all()
                continue
            blo = [max(lo[d], 0) for d in range(3)]
            bhi = [min(hi[d], n3[d]) for d in range(3)]
            shape = [bhi[d] - blo[d] for d in range(3)]
            raw = np.zeros(shape, NP[a.dtype])
            H.HDArrayReadDeviceBuffer(a, p, blo[:len(dims)], bhi[:len(dims)], raw)
            G = oa.G.reshape(n3)[blo[0]:bhi[0], blo[1]:bhi[1], blo[2]:bhi[2]]
            hv = have[p].reshape(n3)[blo[0]:bhi[0], blo[1]:bhi[1], blo[2]:bhi[2]].astype(bool)
            # elements held as current that were ever written (never-written ones are zero)
            bad = hv & (raw.view(np.uint8).reshape(shape + [-1]) != G.view(np.uint8).reshape(shape + [-1])).any(-1)
            assert not bad.any(), "device %d of %s: %d current elements differ" % (p, name, bad.sum())
            # everything outside the device's buffer must be stale or never written
            outside = np.ones(n3, bool)
            outside[blo[0]:bhi[0], blo[1]:bhi[1], blo[2]:bhi[2]] = False
            held_out = have[p].reshape(n3).astype(bool) & outside & (owner.reshape(n3) >= 0)
            assert not held_out.any()


def run_program(prog, ndev, values, gpu_lib, check_buffers=True, mode=H.HDARRAY_MODE_FUSED, setup=None):
    gpu_lib(ndev)
    H.HDArraySetMode(mode)
    if setup:
        setup()
    lib = LibraryRun(H, ndev)
    lib_out = lib.run(prog, values)
    orc = OracleRun(ndev)
    orc_out = orc.run(prog, values)
    dims = {op[1]: tuple(op[3]) for op in prog if op[0] == "create"}
    n = compare_messages(orc_out, lib_out, prog, dims, ndev)
    if check_buffers:
        device_buffers_match(lib, orc, list(dims))
    return lib, orc, lib_out, orc_out, n


def jacobi_prog(dims, P, iters, ptype=ROW, dtype="float", pingpong=True):
    nd = len(dims)
    kernel = "jacobi2d" if nd == 2 else "stencil3d"
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
    return prog, x


def read_all(lib, name, dims, dtype, part="D"):
    out = np.zeros(dims, NP[dtype])
    H.HDArrayRead(lib.arrays[name], out, lib.parts[part])
    return out


# ---------------------------------------------------------------------------------------------
# Jacobi 2-D
# ---------------------------------------------------------------------------------------------

CASES = [
    ((130, 301), 4, BLOCK, "float", True),
    ((97, 131), 3, ROW, "double", False),
    ((140, 270), 5, COL, "bf16", True),
    ((259, 515), 6, BLOCK, "float", False),
    ((70, 600), 2, ROW, "bf16", False),
    ((300, 90), 7, ROW, "double", True),
]


@pytest.mark.parametrize("dims,P,ptype,dtype,pingpong", CASES)
@pytest.mark.parametrize("mode", [H.HDARRAY_MODE_FUSED, H.HDARRAY_MODE_PLAIN])
def test_jacobi2d_parity(gpu_lib, dims, P, ptype, dtype, pingpong, mode):
    x = synthetic.jacobi_field(dims, stream=11, dtype=dtype)
    prog, last = jacobi_prog(dims, P, 5, ptype, dtype, pingpong)
    lib, orc, *_ = run_program(prog, P, {"B": x, "A": x}, gpu_lib, mode=mode)
    got = read_all(lib, last, dims, dtype)
    want = orc.arrays[last].G
    assert np.array_equal(got.view(np.uint8), want.view(np.uint8))


def test_jacobi2d_tile_shapes(gpu_lib, monkeypatch):
    """Tiles of several heights, a ragged last band and 1-row partitions."""
    dims, P = (41, 1030), 13  # 39 work rows over 13 devices: 3 rows each
    x = synthetic.jacobi_field(dims, stream=12, dtype="float")
    prog, last = jacobi_prog(dims, P, 4, ROW, "float", True)
    lib, orc, *_ = run_program(prog, P, {"B": x, "A": x}, gpu_lib)
    assert np.array_equal(read_all(lib, last, dims, "float"), orc.arrays[last].G)


def test_jacobi2d_degenerate(gpu_lib):
    """3x3 array (one work element), more devices than work rows (idle devices)."""
    for dims, P in (((3, 3), 1), ((3, 9), 4), ((9, 3), 5)):
        x = synthetic.jacobi_field(dims, stream=13, dtype="double")
        prog, last = jacobi_prog(dims, P, 3, ROW, "double", False)
        lib, orc, *_ = run_program(prog, P, {"B": x, "A": x}, gpu_lib)
        assert np.array_equal(read_all(lib, last, dims, "double"), orc.arrays[last].G)
        H.HDArrayExit()


def test_empty_work_region(gpu_lib):
    """A call over a partition whose work region is empty moves nothing, launches nothing and
    leaves the arrays as they were; zero-size arrays are refused."""
    dims, P = (40, 56), 4
    gpu_lib(P)
    x = synthetic.jacobi_field(dims, stream=14, dtype="float")
    B = H.HDArrayCreate("B", "float", None, *dims)
    A = H.HDArrayCreate("A", "float", None, *dims)
    D = H.HDArrayPartition(ROW, dims, (0, 0), dims, P)
    E = H.HDArrayPartition(ROW, dims, (5, 1), (5, dims[1] - 1), P)  # no rows
    H.HDArrayWrite(B, x, D)
    H.HDArrayWrite(A, x, D)
    c0 = H.HDArrayGetCounters()
    H.HDArrayApplyKernel("jacobi2d", E, B, A)
    c1 = H.HDArrayGetCounters()
    assert c1["launches"] == c0["launches"]
    assert H.HDArrayGetPlan(B) == []
    got = np.zeros(dims, np.float32)
    H.HDArrayRead(A, got, D)
    assert np.array_equal(got, x)
    for bad in ((0, 5), (5, 0)):
        with pytest.raises(H.HDArrayError):
            H.HDArrayCreate("Z", "float", None, *bad)


def test_tune_cache_file(gpu_lib, monkeypatch, tmp_path):
    """Autotuning with HDARRAY_TUNE_CACHE: the first run times the candidates and appends the
    chosen shape (key and nine integers); after a new HDArrayInit the shape comes from the file,
    nothing is appended, and the results stay bit-exact against the oracle."""
    cache = tmp_path / "tune.txt"
    monkeypatch.setenv("HDARRAY_AUTOTUNE", "1")
    monkeypatch.setenv("HDARRAY_TUNE_CACHE", str(cache))
    dims, P = (300, 260), 4
    x = synthetic.jacobi_field(dims, stream=15, dtype="float")
    prog, last = jacobi_prog(dims, P, 6, BLOCK, "float", True)
    lib, orc, *_ = run_program(prog, P, {"B": x, "A": x}, gpu_lib)
    assert np.array_equal(read_all(lib, last, dims, "float"), orc.arrays[last].G)
    lines = cache.read_text().splitlines()
    assert lines and all(len(ln.split()) == 10 for ln in lines)
    H.HDArrayExit()
    lib, orc, *_ = run_program(prog, P, {"B": x, "A": x}, gpu_lib)
    assert np.array_equal(read_all(lib, last, dims, "float"), orc.arrays[last].G)
    assert cache.read_text().splitlines() == lines


# ---------------------------------------------------------------------------------------------
# Reduce, residual
# ---------------------------------------------------------------------------------------------

@pytest.mark.parametrize("dtype", ["double", "float", "bf16"])
def test_reduce_parity(gpu_lib, dtype):
    dims, P = (203, 157), 6
    u = synthetic.uniform(dims[0] * dims[1], stream=21).reshape(dims)
    x = synthetic.to_storage(1.0 + (u - 0.5) * 0.02, dtype)  # products stay well scaled
    prog = [("create", "X", dtype, dims), ("part", "D", BLOCK, dims, (0, 0), dims, P),
            ("part", "C", COL, dims, (2, 3), (dims[0] - 5, dims[1] - 1), 4),
            ("write", "X", "D")]
    for op in (0, 1, 2, 3):
        prog.append(("reduce", "X", op, "C"))
        prog.append(("reduce", "X", op, "D"))
    lib, orc, lib_out, orc_out, _ = run_program(prog, P, {"X": x}, gpu_lib)
    for lo, oo, op in zip(lib_out, orc_out, prog):
        if op[0] != "reduce":
            continue
        g, w = lo["_value"], oo["_value"]
        if op[2] in (2, 3):
            assert g == w
        elif op[2] == 0:
            assert abs(g - w) <= 1e-12 * abs(w)
        else:
            assert w > 1e-3 and abs(g - w) <= 4 * dims[0] * dims[1] * 2.0 ** -53 * abs(w)


def test_residual_flow_cfg1(gpu_lib):
    """The paper's two-kernel Jacobi (plain form, FP64, 256x256, ROW 4, 10 iterations) and the
    FP64 residual sum((A - B)^2) via HDArrayReduce."""
    dims, P = (256, 256), 4
    x = synthetic.jacobi_field(dims, stream=0, dtype="double")
    prog, _ = jacobi_prog(dims, P, 10, ROW, "double", pingpong=False)
    # the residual of the last step, between the new iterate A and the old B (before the copy back)
    prog = prog[:-1] + [("create", "R", "double", dims), ("apply", "sqdiff", "W", ["A", "B", "R"]),
                        ("reduce", "R", 0, "W"), prog[-1]]
    lib, orc, lib_out, orc_out, _ = run_program(prog, P, {"B": x, "A": x}, gpu_lib,
                                                mode=H.HDARRAY_MODE_PLAIN)
    g, w = lib_out[-2]["_value"], orc_out[-2]["_value"]
    assert w > 0 and abs(g - w) <= 1e-12 * abs(w)


@pytest.mark.parametrize("dims,P,ptype,dtype", [((203, 157), 6, BLOCK, "float"), ((131, 267), 5, COL, "bf16"),
                                              ((97, 141), 3, ROW, "double"), ((37, 45, 61), 4, COL, "float")])
def test_residual_fused_sum(gpu_lib, dims, P, ptype, dtype):
    """The fused form's residual: R = (X - Y)^2 stored bit-exact on every device, and
    HDArrayReduce(R, SUM) over the residual's own boxes (the sum the residual launch folded) and
    over another partition (a separate fold of R) both within 1e-12 of the oracle, also after R is
    redefined by a second residual.  The partitions' odd boundaries put rows at every 16-byte
    phase, so the kernel's scalar heads and tails and its vectors are all exercised."""
    nd = len(dims)
    n = int(np.prod(dims))
    x = synthetic.to_storage(synthetic.uniform(n, stream=31).reshape(dims), dtype)
    y = synthetic.to_storage(synthetic.uniform(n, stream=32).reshape(dims), dtype)
    z = synthetic.to_storage(synthetic.uniform(n, stream=33).reshape(dims), dtype)
    prog = [("create", "X", dtype, dims), ("create", "Y", dtype, dims), ("create", "Z", dtype, dims),
            ("create", "R", "double", dims),
            ("part", "D", ptype, dims, (0,) * nd, dims, P),
            ("part", "W", ptype, dims, (1,) * nd, tuple(k - 2 for k in dims), P),
            ("part", "V", ROW, dims, (1,) * nd, tuple(k - 2 for k in dims), 2),
            ("write", "X", "D"), ("write", "Y", "D"), ("write", "Z", "D"),
            ("apply", "sqdiff", "W", ["X", "Y", "R"]),
            ("reduce", "R", 0, "W"), ("reduce", "R", 0, "W"), ("reduce", "R", 0, "V"),
            ("apply", "sqdiff", "W", ["Z", "Y", "R"]),
            ("reduce", "R", 0, "W"), ("reduce", "R", 2, "W")]
    lib, orc, lib_out, orc_out, _ = run_program(prog, P, {"X": x, "Y": y, "Z": z}, gpu_lib)
    nred = 0
    for lo, oo, op in zip(lib_out, orc_out, prog):
        if op[0] != "reduce":
            continue
        g, w = lo["_value"], oo["_value"]
        assert w > 0
        assert (g == w) if op[2] == 2 else abs(g - w) <= 1e-12 * abs(w), (op, g, w)
        nred += 1
    assert nred == 5


def test_residual_sum_follows_graph_replays(gpu_lib):
    """A residual recorded in a graph: every replay redefines R, so HDArrayReduce after the
    replays folds the replays' values (the sum kept from the recorded call is not reused), and
    the result matches the oracle after the same calls."""
    torch = pytest.importorskip("torch")
    dims, P, dtype = (150, 211), 4, "float"
    x = synthetic.jacobi_field(dims, stream=34, dtype=dtype)
    gpu_lib(P)
    B = H.HDArrayCreate("B", dtype, None, *dims)
    A = H.HDArrayCreate("A", dtype, None, *dims)
    R = H.HDArrayCreate("R", "double", None, *dims)
    D = H.HDArrayPartition(BLOCK, dims, (0, 0), dims, P)
    W = H.HDArrayPartition(BLOCK, dims, (1, 1), (dims[0] - 1, dims[1] - 1), P)
    H.HDArrayWrite(B, x, D)
    for _ in range(2):
        H.HDArrayApplyKernel("jacobi2d", W, B, A)
        H.HDArrayApplyKernel("jacobi2d", W, A, B)
    H.HDArrayApplyKernel("sqdiff", W, B, A, R)  # R defined before the recording: a periodic graph
    H.HDArrayGraphBegin()
    H.HDArrayApplyKernel("jacobi2d", W, B, A)
    H.HDArrayApplyKernel("jacobi2d", W, A, B)
    H.HDArrayApplyKernel("sqdiff", W, B, A, R)
    gid = H.HDArrayGraphEnd()
    H.HDArrayGraphLaunch(gid, 3)
    got = H.HDArrayReduce(R, 0, W)
    torch.cuda.synchronize()
    o = oracle.Oracle(P)
    ob, oa = o.create("B", dtype, dims), o.create("A", dtype, dims)
    orr = o.create("R", "double", dims)
    od = o.partition(BLOCK, dims, (0, 0), dims)
    ow = o.partition(BLOCK, dims, (1, 1), (dims[0] - 1, dims[1] - 1))
    o.write(ob, x, od)
    for i in range(2 + 1 + 3):  # warm-up, recording, three replays
        o.apply("jacobi2d", ow, [ob, oa])
        o.apply("jacobi2d", ow, [oa, ob])
        if i >= 1:
            o.apply("sqdiff", ow, [ob, oa, orr])
    want, _ = o.reduce(orr, 0, ow)
    assert want > 0 and abs(got - want) <= 1e-12 * want


@pytest.mark.parametrize("async_write", ["1", "0"])
def test_write_from_pinned_memory_is_ordered(gpu_lib, monkeypatch, async_write):
    """HDArrayWrite from pinned host memory into existing buffers runs on the library's copy
    stream (HDARRAY_ASYNC_WRITE=1): every later use of the array waits for it, and it waits for
    the library's earlier work on that array -- here a Write right after a kernel that reads the
    array, and Writes of one input while the other is being computed on.  Results equal the
    oracle's after the same calls, bit for bit, with the copy stream and without it."""
    torch = pytest.importorskip("torch")
    monkeypatch.setenv("HDARRAY_ASYNC_WRITE", async_write)
    dims, P, dtype = (1030, 770), 4, "float"
    xs = [synthetic.jacobi_field(dims, stream=35 + i, dtype=dtype) for i in range(3)]
    pinned = [torch.from_numpy(x).pin_memory() for x in xs]
    gpu_lib(P)
    B0 = H.HDArrayCreate("B0", dtype, None, *dims)
    B1 = H.HDArrayCreate("B1", dtype, None, *dims)
    A = H.HDArrayCreate("A", dtype, None, *dims)
    D = H.HDArrayPartition(BLOCK, dims, (0, 0), dims, P)
    W = H.HDArrayPartition(BLOCK, dims, (1, 1), (dims[0] - 1, dims[1] - 1), P)
    o = oracle.Oracle(P)
    ob = [o.create("B0", dtype, dims), o.create("B1", dtype, dims)]
    oa = o.create("A", dtype, dims)
    od = o.partition(BLOCK, dims, (0, 0), dims)
    ow = o.partition(BLOCK, dims, (1, 1), (dims[0] - 1, dims[1] - 1))
    lb = [B0, B1]
    for i in range(2):  # first Writes allocate the buffers
        H.HDArrayWrite(lb[i], pinned[i], D)
        o.write(ob[i], xs[i], od)
    H.HDArrayApplyKernel("jacobi2d", W, lb[0], A)
    o.apply("jacobi2d", ow, [ob[0], oa])
    for k in range(6):
        cur, nxt = k % 2, (k + 1) % 2
        H.HDArrayApplyKernel("jacobi2d", W, A, lb[cur])         # reads A, writes B_cur
        o.apply("jacobi2d", ow, [oa, ob[cur]])
        H.HDArrayWrite(lb[nxt], pinned[(k + 2) % 3], D)           # the other input, while B_cur is used
        o.write(ob[nxt], xs[(k + 2) % 3], od)
        H.HDArrayApplyKernel("jacobi2d", W, lb[cur], A)          # reads B_cur
        o.apply("jacobi2d", ow, [ob[cur], oa])
        H.HDArrayWrite(lb[cur], pinned[k % 3], D)                 # overwrites B_cur right after that read
        o.write(ob[cur], xs[k % 3], od)
        H.HDArrayApplyKernel("jacobi2d", W, lb[nxt], A)
        o.apply("jacobi2d", ow, [ob[nxt], oa])
    for h, oarr in ((A, oa), (B0, ob[0]), (B1, ob[1])):
        got = np.zeros(dims, np.float32)
        H.HDArrayRead(h, got, D)
        assert np.array_equal(got, oarr.G)


# ---------------------------------------------------------------------------------------------
# GEMM (binary64)
# ---------------------------------------------------------------------------------------------

def _gamma_bound(A, B, C0, alpha, beta, k):
    u = 2.0 ** -53
    gam = (k + 2) * u / (1 - (k + 2) * u)
    return gam * (np.abs(beta * C0) + abs(alpha) * (np.abs(A) @ np.abs(B))) + 1e-300


@pytest.mark.parametrize("mode", [H.HDARRAY_MODE_FUSED, H.HDARRAY_MODE_PLAIN])
def test_gemm_listing2_parity(gpu_lib, mode):
    ni, nj, nk, P = 150, 130, 170, 4
    a = synthetic.normal(ni * nk, stream=31).reshape(ni, nk)
    b = synthetic.normal(nk * nj, stream=32).reshape(nk, nj)
    c = synthetic.normal(ni * nj, stream=33).reshape(ni, nj)
    alpha, beta = 1.5, 0.25
    prog = [("create", "a", "double", (ni, nk)), ("create", "b", "double", (nk, nj)),
            ("create", "c", "double", (ni, nj)),
            ("part", "p0", ROW, (ni, nj), (0, 0), (ni, nj), P),
            ("part", "pa", ROW, (ni, nk), (0, 0), (ni, nk), P),
            ("part", "pb", ROW, (nk, nj), (0, 0), (nk, nj), P),
            ("write", "a", "pa"), ("write", "b", "pb"), ("write", "c", "p0"),
            ("apply", "gemm", "p0", ["a", "b", "c"], (alpha, beta, ni, nj, nk))]
    lib, orc, *_ = run_program(prog, P, {"a": a, "b": b, "c": c}, gpu_lib, check_buffers=False, mode=mode)
    device_buffers_match(lib, orc, ["a", "b"])  # the all-gathered B is bit-exact on every device
    got = np.zeros((ni, nj))
    H.HDArrayRead(lib.arrays["c"], got, lib.parts["p0"])
    want = orc.arrays["c"].G
    assert (np.abs(got - want) <= 2 * _gamma_bound(a, b, c, alpha, beta, nk)).all()


def test_trmm_trapezoid_parity(gpu_lib):
    n, m, P = 256, 96, 4
    a, b = synthetic.tri_gemm_inputs(n, m, stream=34)
    rows = [p * n // P for p in range(P + 1)]
    prog = [("create", "A", "double", (n, n)), ("create", "B", "double", (n, m)),
            ("create", "C", "double", (n, m)),
            ("part", "R", ROW, (n, m), (0, 0), (n, m), P),
            ("part", "RA", ROW, (n, n), (0, 0), (n, n), P)]
    for p in range(P):
        r0, r1 = rows[p], rows[p + 1]
        prog.append(("trap_use", "trmm", "R", "A", p, (r0, 0, r0, r0, r1 - 1, 0, r1 - 1, r1 - 1)))
    prog += [("write", "A", "RA"), ("write", "B", "R"),
             ("apply", "trmm", "R", ["A", "B", "C"], (1.0, 0.0)),
             ("apply", "trmm", "R", ["A", "B", "C"], (1.0, 0.0))]
    lib, orc, lib_out, *_ = run_program(prog, P, {"A": a, "B": b}, gpu_lib, check_buffers=False)
    device_buffers_match(lib, orc, ["A", "B"])
    got = np.zeros((n, m))
    H.HDArrayRead(lib.arrays["C"], got, lib.parts["R"])
    assert (np.abs(got - orc.arrays["C"].G) <= 2 * _gamma_bound(np.tril(a), b, 0 * got, 1.0, 0.0, n)).all()


# ---------------------------------------------------------------------------------------------
# batches and graphs
# ---------------------------------------------------------------------------------------------

def test_batch_of_instances(gpu_lib):
    insts = synthetic.jacobi_instances(9, stream=41, lo=8, hi=200)
    ndev = max(p for _, _, p, _ in insts)
    gpu_lib(ndev)
    arrays = []
    xs = []
    for i, (r, c, P, kind) in enumerate(insts):
        t = ROW if kind == "ROW" else COL
        x = synthetic.jacobi_field((r, c), stream=100 + i, dtype="float")
        B = H.HDArrayCreate("B%d" % i, "float", None, r, c)
        A = H.HDArrayCreate("A%d" % i, "float", None, r, c)
        D = H.HDArrayPartition(t, (r, c), (0, 0), (r, c), P)
        W = H.HDArrayPartition(t, (r, c), (1, 1), (r - 1, c - 1), P)
        H.HDArrayWrite(B, x, D)
        H.HDArrayWrite(A, x, D)
        arrays.append([B, A, D, W])
        xs.append(x)
    iters = 6
    for it in range(iters):
        H.HDArrayBatchBegin()
        for B, A, D, W in arrays:
            H.HDArrayApplyKernel("jacobi2d", W, B, A)
        H.HDArrayBatchEnd()
        for inst in arrays:
            inst[0], inst[1] = inst[1], inst[0]
    for i, ((r, c, P, kind), (B, A, D, W)) in enumerate(zip(insts, arrays)):
        got = np.zeros((r, c), np.float32)
        H.HDArrayRead(B, got, D)
        o = oracle.Oracle(P)
        t = ROW if kind == "ROW" else COL
        ob, oa = o.create("B", "float", (r, c)), o.create("A", "float", (r, c))
        od = o.partition(t, (r, c), (0, 0), (r, c))
        ow = o.partition(t, (r, c), (1, 1), (r - 1, c - 1))
        o.write(ob, xs[i], od)
        o.write(oa, xs[i], od)
        for it in range(iters):
            o.apply("jacobi2d", ow, [ob, oa])
            ob, oa = oa, ob
        assert np.array_equal(got, ob.G), "instance %d" % i


def test_batch_rejects_dependent_calls(gpu_lib):
    gpu_lib(2)
    B = H.HDArrayCreate("B", "float", None, 16, 16)
    A = H.HDArrayCreate("A", "float", None, 16, 16)
    W = H.HDArrayPartition(ROW, (16, 16), (1, 1), (15, 15), 2)
    H.HDArrayBatchBegin()
    H.HDArrayApplyKernel("jacobi2d", W, B, A)
    with pytest.raises(H.HDArrayError) as e:
        H.HDArrayApplyKernel("jacobi2d", W, A, B)  # uses what the first call defines
    assert e.value.code == -3
    H.HDArrayBatchEnd()  # the first call still runs


@pytest.mark.parametrize("dtype", ["float", "bf16"])
def test_graph_replay(gpu_lib, dtype):
    dims, P = (200, 330), 6
    x = synthetic.jacobi_field(dims, stream=51, dtype=dtype)
    gpu_lib(P)
    B = H.HDArrayCreate("B", dtype, None, *dims)
    A = H.HDArrayCreate("A", dtype, None, *dims)
    D = H.HDArrayPartition(BLOCK, dims, (0, 0), dims, P)
    W = H.HDArrayPartition(BLOCK, dims, (1, 1), (dims[0] - 1, dims[1] - 1), P)
    H.HDArrayWrite(B, x, D)
    H.HDArrayWrite(A, x, D)
    for _ in range(2):  # reach the periodic state
        H.HDArrayApplyKernel("jacobi2d", W, B, A)
        H.HDArrayApplyKernel("jacobi2d", W, A, B)
    H.HDArrayGraphBegin()
    H.HDArrayApplyKernel("jacobi2d", W, B, A)
    H.HDArrayApplyKernel("jacobi2d", W, A, B)
    gid = H.HDArrayGraphEnd()
    H.HDArrayGraphLaunch(gid, 7)
    total = 2 * 2 + 2 + 2 * 7
    got = np.zeros(dims, NP[dtype])
    H.HDArrayRead(B, got, D)
    o = oracle.Oracle(P)
    ob, oa = o.create("B", dtype, dims), o.create("A", dtype, dims)
    od = o.partition(BLOCK, dims, (0, 0), dims)
    ow = o.partition(BLOCK, dims, (1, 1), (dims[0] - 1, dims[1] - 1))
    o.write(ob, x, od)
    o.write(oa, x, od)
    for _ in range(total // 2):
        o.apply("jacobi2d", ow, [ob, oa])
        o.apply("jacobi2d", ow, [oa, ob])
    assert np.array_equal(got, ob.G)
    # a graph recorded in another state refuses to run
    H.HDArrayApplyKernel("jacobi2d", W, B, A)
    with pytest.raises(H.HDArrayError) as e:
        H.HDArrayGraphLaunch(gid, 1)
    assert e.value.code == -7


# ---------------------------------------------------------------------------------------------
# full size, in the benchmark's configuration: sampled outputs against the oracle
# ---------------------------------------------------------------------------------------------

# tile shapes: the library's defaults, and the shapes the autotuner picks for bench.py on a GB300
TUNED_2D = {"float": {"HDARRAY_JACOBI_VARIANT": "5", "HDARRAY_TILE_ROWS": "8", "HDARRAY_BAND2": "64"},
            "bf16": {"HDARRAY_JACOBI_VARIANT": "3", "HDARRAY_TILE_ROWS": "16", "HDARRAY_BAND2": "32"}}
TMA_2D = {"HDARRAY_JACOBI_VARIANT": "5", "HDARRAY_TILE_ROWS": "16", "HDARRAY_BAND2": "32"}


@pytest.mark.parametrize("tuned", [False, True, "tma"])
@pytest.mark.parametrize("dtype", ["float", "bf16"])
def test_full_size_8192_block16_graph(gpu_lib, dtype, tuned, monkeypatch):
    """The benchmark workload (8192^2, BLOCK 4 x 4, a 2-iteration graph replayed to 100
    iterations) with the default tile shape and with the one bench.py runs after autotuning."""
    for k, v in (TMA_2D.items() if tuned == "tma" else TUNED_2D[dtype].items() if tuned else ()):
        monkeypatch.setenv(k, v)
    n, P, T = 8192, 16, 100
    dims = (n, n)
    x = synthetic.jacobi_field(dims, stream=1, dtype=dtype)
    gpu_lib(P)
    B = H.HDArrayCreate("B", dtype, None, n, n)
    A = H.HDArrayCreate("A", dtype, None, n, n)
    D = H.HDArrayPartition(BLOCK, dims, (0, 0), dims, P)
    W = H.HDArrayPartition(BLOCK, dims, (1, 1), (n - 1, n - 1), P)
    H.HDArrayWrite(B, x, D)
    H.HDArrayWrite(A, x, D)
    for _ in range(2):
        H.HDArrayApplyKernel("jacobi2d", W, B, A)
        H.HDArrayApplyKernel("jacobi2d", W, A, B)
    H.HDArrayGraphBegin()
    H.HDArrayApplyKernel("jacobi2d", W, B, A)
    H.HDArrayApplyKernel("jacobi2d", W, A, B)
    gid = H.HDArrayGraphEnd()
    H.HDArrayGraphLaunch(gid, (T - 6) // 2)
    got = np.zeros(dims, NP[dtype])
    H.HDArrayRead(B, got, D)
    rng = np.random.default_rng(7)
    cuts = [1, 2, 2047, 2048, 2049, 4096, 4097, 6143, 6144, 8190]
    samples = [(int(rng.integers(0, n)), int(rng.integers(0, n))) for _ in range(24)]
    samples += [(c, int(rng.integers(0, n))) for c in cuts] + [(int(rng.integers(0, n)), c) for c in cuts]
    samples += [(0, 0), (8191, 8191), (1, 1), (8190, 8190), (2048, 2048)]
    prec = {"float": 1, "bf16": 2}[dtype]
    want = light_cone(x, prec, samples, T)
    gotv = np.array([got[i, j] for i, j in samples])
    assert np.array_equal(gotv.view(np.uint8), want.view(np.uint8))
    # accuracy against binary64 on the same samples
    x64 = synthetic.jacobi_field(dims, stream=1, dtype="double")
    ref = light_cone(x64, 0, samples, T)
    vals = gotv.astype(np.float64) if dtype == "float" else oracle.bf16_to_f32(gotv).astype(np.float64)
    if dtype == "float":
        assert np.abs(vals - ref).max() / np.abs(ref).max() <= 1e-5
    else:
        # one rounding to bfloat16 per step, each at most 2^-9 of the field's maximum, and the
        # Jacobi average does not amplify errors: after T steps the error is at most T * 2^-9 * max|x0|
        assert np.abs(vals - ref).max() <= T * 2.0 ** -9 * np.abs(x64).max()


# ---------------------------------------------------------------------------------------------
# 3-D 7-point stencil on uneven manual partitions
# ---------------------------------------------------------------------------------------------

def stencil3d_prog(n, boxes, iters, dtype):
    work = [(tuple(max(1, v) for v in lo), tuple(min(n - 1, v) for v in hi)) for lo, hi in boxes]
    dims = (n, n, n)
    prog = [("create", "B", dtype, dims), ("create", "A", dtype, dims),
            ("manual", "D", dims, boxes), ("manual", "W", dims, work),
            ("write", "B", "D")]
    x, y = "B", "A"
    for _ in range(iters):
        prog.append(("apply", "stencil3d", "W", [x, y]))
        x, y = y, x
    return prog, x


@pytest.mark.parametrize("dtype", ["float", "double", "bf16"])
@pytest.mark.parametrize("mode", [H.HDARRAY_MODE_FUSED, H.HDARRAY_MODE_PLAIN])
def test_stencil3d_parity(gpu_lib, dtype, mode):
    n = 40
    boxes = synthetic.kd_boxes(n, 9, stream=61, min_ext=6, max_ext=40)
    x = synthetic.jacobi_field((n, n, n), stream=62, dtype=dtype)
    prog, last = stencil3d_prog(n, boxes, 4, dtype)
    lib, orc, *_ = run_program(prog, len(boxes), {"B": x}, gpu_lib, mode=mode)
    got = np.zeros((n, n, n), NP[dtype])
    H.HDArrayRead(lib.arrays[last], got, lib.parts["D"])
    assert np.array_equal(got.view(np.uint8), orc.arrays[last].G.view(np.uint8))


def test_stencil3d_wide_rows(gpu_lib):
    """Boxes wider than one band (several x bands per row) and ragged z chunks."""
    n = 70
    dims = (n, n, 300)
    boxes = [((0, 0, 0), (35, 70, 130)), ((0, 0, 130), (35, 70, 300)), ((35, 0, 0), (70, 33, 300)),
             ((35, 33, 0), (70, 70, 300))]
    work = [(tuple(max(1, v) for v in lo), tuple(min(d - 1, v) for v, d in zip(hi, dims))) for lo, hi in boxes]
    x = synthetic.jacobi_field(dims, stream=63, dtype="float")
    prog = [("create", "B", "float", dims), ("create", "A", "float", dims),
            ("manual", "D", dims, boxes), ("manual", "W", dims, work), ("write", "B", "D"),
            ("apply", "stencil3d", "W", ["B", "A"]), ("apply", "stencil3d", "W", ["A", "B"]),
            ("apply", "stencil3d", "W", ["B", "A"])]
    lib, orc, *_ = run_program(prog, 4, {"B": x}, gpu_lib)
    got = np.zeros(dims, np.float32)
    H.HDArrayRead(lib.arrays["A"], got, lib.parts["D"])
    assert np.array_equal(got, orc.arrays["A"].G)


@pytest.mark.parametrize("tile_z,variant", [(None, None), ("32", None), ("32", "3")])
def test_full_size_stencil3d_512_37_boxes(gpu_lib, tile_z, variant, monkeypatch):
    """512^3 on the 37 k-d boxes, 50 iterations in a graph, with the default tile depth and the
    one bench.py's autotuner picks (32 planes), planes staged by cp.async or by bulk tensor copies."""
    if tile_z:
        monkeypatch.setenv("HDARRAY_TILE_Z", tile_z)
    if variant:
        monkeypatch.setenv("HDARRAY_STENCIL3D_VARIANT", variant)
    n, T = 512, 50
    boxes = synthetic.kd_boxes(n, 37, stream=3)
    x = synthetic.jacobi_field((n, n, n), stream=3, dtype="float")
    gpu_lib(37)
    B = H.HDArrayCreate("B", "float", None, n, n, n)
    A = H.HDArrayCreate("A", "float", None, n, n, n)
    D = H.HDArrayPartitionManual((n, n, n), boxes)
    work = [(tuple(max(1, v) for v in lo), tuple(min(n - 1, v) for v in hi)) for lo, hi in boxes]
    W = H.HDArrayPartitionManual((n, n, n), work)
    H.HDArrayWrite(B, x, D)
    for _ in range(2):
        H.HDArrayApplyKernel("stencil3d", W, B, A)
        H.HDArrayApplyKernel("stencil3d", W, A, B)
    H.HDArrayGraphBegin()
    H.HDArrayApplyKernel("stencil3d", W, B, A)
    H.HDArrayApplyKernel("stencil3d", W, A, B)
    gid = H.HDArrayGraphEnd()
    H.HDArrayGraphLaunch(gid, (T - 6) // 2)
    got = np.zeros((n, n, n), np.float32)
    H.HDArrayRead(B, got, D)
    rng = np.random.default_rng(9)
    samples = [tuple(int(v) for v in rng.integers(0, n, 3)) for _ in range(6)]
    for lo, hi in boxes[:6]:  # box corners and faces: T-junctions of uneven partitions
        samples.append((lo[0], min(hi[1], n - 1), lo[2]))
        samples.append((min(hi[0], n - 1) - 1, lo[1], max(lo[2] - 1, 0)))
    samples += [(0, 0, 0), (1, 1, 1), (510, 510, 510)]
    want = light_cone3(x, 1, samples, T)
    gotv = np.array([got[s] for s in samples])
    assert np.array_equal(gotv, want)


# ---------------------------------------------------------------------------------------------
# GEMM on binary32 arrays: tensor cores with the bf16x3 split
# ---------------------------------------------------------------------------------------------

def _bf16x3_bound(A, B, C0, alpha, beta, k):
    """Componentwise bound for the bf16x3 product in binary32: each operand x = hi + lo + d with
    |d| <= 2^-16 |x| and |lo| <= 2^-8 |x|, so dropping lo*lo and the two d terms loses at most
    3 * 2^-16 |a||b| per product; binary32 accumulation of k terms adds (k + 2) * 2^-24."""
    A64, B64 = A.astype(np.float64), B.astype(np.float64)
    mag = abs(alpha) * (np.abs(A64) @ np.abs(B64)) + abs(beta) * np.abs(C0.astype(np.float64))
    return (3 * 2.0 ** -16 + (k + 2) * 2.0 ** -24) * mag + 1e-30


def _bf16x6_bound(A, B, C0, alpha, beta, k):
    """Componentwise bound for the bf16x6 product: x = hi + mid + lo + d with |d| <= 2^-24 |x|,
    |mid| <= 2^-8 |x|, |lo| <= 2^-16 |x|; the kept products miss d and mid*lo, lo*mid, lo*lo, at
    most 4 * 2^-24 |a||b| per product, and six binary32 accumulations per k step add
    (6k + 2) * 2^-24."""
    A64, B64 = A.astype(np.float64), B.astype(np.float64)
    mag = abs(alpha) * (np.abs(A64) @ np.abs(B64)) + abs(beta) * np.abs(C0.astype(np.float64))
    return (4 * 2.0 ** -24 + (6 * k + 2) * 2.0 ** -24) * mag + 1e-30, mag


@pytest.mark.parametrize("panels,split", [(True, 2), (False, 2), (True, 3)])
@pytest.mark.parametrize("shape,P,lower", [((200, 300, 150), 2, False), ((512, 256, 512), 4, True),
                                            ((384, 520, 384), 3, True)])
def test_gemm_bf16x3_parity(gpu_lib, shape, P, lower, panels, split, monkeypatch):
    """split 2: bf16x3 within its componentwise bound; split 3: bf16x6 within its bound and within
    1e-5 of |A||B| componentwise (binary32 accuracy)."""
    if not panels:  # the fallback kernel that splits while loading
        monkeypatch.setenv("HDARRAY_GEMM_NO_PANELS", "1")
    ni, nj, nk = shape
    if lower:
        a, b = synthetic.tri_gemm_inputs(ni, nj, stream=71, dtype="float")
    else:
        a = synthetic.to_storage(synthetic.normal(ni * nk, stream=72).reshape(ni, nk), "float")
        b = synthetic.to_storage(synthetic.normal(nk * nj, stream=73).reshape(nk, nj), "float")
    c = synthetic.to_storage(synthetic.normal(ni * nj, stream=74).reshape(ni, nj), "float")
    alpha, beta = (1.0, 0.0) if lower else (1.25, -0.5)
    kname = "trmm" if lower else "gemm"
    scal = (alpha, beta) if lower else (alpha, beta, ni, nj, nk)
    prog = [("create", "A", "float", (ni, nk)), ("create", "B", "float", (nk, nj)),
            ("create", "C", "float", (ni, nj)),
            ("part", "R", ROW, (ni, nj), (0, 0), (ni, nj), P),
            ("part", "RA", ROW, (ni, nk), (0, 0), (ni, nk), P),
            ("part", "RB", ROW, (nk, nj), (0, 0), (nk, nj), P)]
    if lower:
        bx = oracle.partition_boxes(ROW, P, (ni, nj), (0, 0), (ni, nj))
        for p, (lo, hi) in enumerate(bx):
            r0, r1 = lo[0], hi[0]
            prog.append(("trap_use", "trmm", "R", "A", p, (r0, 0, r0, r0, r1 - 1, 0, r1 - 1, r1 - 1)))
    prog += [("write", "A", "RA"), ("write", "B", "RB"), ("write", "C", "R"),
             ("apply", kname, "R", ["A", "B", "C"], scal)]
    setup = (lambda: H.HDArraySetGemmSplit(H.HDARRAY_GEMM_BF16X6)) if split == 3 else None
    lib, orc, *_ = run_program(prog, P, {"A": a, "B": b, "C": c}, gpu_lib, check_buffers=False, setup=setup)
    device_buffers_match(lib, orc, ["A", "B"])  # the all-gathered B is bit-exact on every device
    got = np.zeros((ni, nj), np.float32)
    H.HDArrayRead(lib.arrays["C"], got, lib.parts["R"])
    # against the oracle: the binary64 product of the stored inputs rounded once to binary32, so
    # one unit in the last place of its result covers that rounding on top of the exact product's
    # bound
    want32 = orc.arrays["C"].G
    want = want32.astype(np.float64)
    ulp = np.spacing(np.abs(want32)).astype(np.float64)
    err = np.abs(got.astype(np.float64) - want)
    if split == 2:
        bound = _bf16x3_bound(np.tril(a) if lower else a, b, c, alpha, beta, nk)
        assert (err <= 2 * bound + ulp).all(), float((err / (bound + ulp)).max())
    else:
        bound, mag = _bf16x6_bound(np.tril(a) if lower else a, b, c, alpha, beta, nk)
        assert (err <= bound + ulp).all(), float((err / (bound + ulp)).max())
        assert (err <= 1e-5 * mag + ulp).all(), float((err / mag).max())
    # the oracle's result is the binary32 rounding of the product numpy computes in binary64 (up
    # to the two binary64 summation orders)
    ref = beta * c.astype(np.float64) + alpha * (np.tril(a.astype(np.float64)) if lower else a.astype(np.float64)) @ b.astype(np.float64)
    mag64 = abs(beta) * np.abs(c.astype(np.float64)) + abs(alpha) * (
        np.abs(np.tril(a.astype(np.float64)) if lower else a.astype(np.float64)) @ np.abs(b.astype(np.float64)))
    assert (np.abs(want - ref) <= ulp + 2 * (nk + 2) * 2.0 ** -53 * mag64).all()


def test_gemm_bf16x3_reuses_panels(gpu_lib):
    """A second call with unchanged A and B reuses the split panels; changing B re-splits it."""
    ni = nj = nk = 256
    a = synthetic.to_storage(synthetic.normal(ni * nk, stream=75).reshape(ni, nk), "float")
    b = synthetic.to_storage(synthetic.normal(nk * nj, stream=76).reshape(nk, nj), "float")
    b2 = synthetic.to_storage(synthetic.normal(nk * nj, stream=77).reshape(nk, nj), "float")
    gpu_lib(2)
    A = H.HDArrayCreate("A", "float", None, ni, nk)
    B = H.HDArrayCreate("B", "float", None, nk, nj)
    C = H.HDArrayCreate("C", "float", None, ni, nj)
    R = H.HDArrayPartition(ROW, (ni, nj), (0, 0), (ni, nj), 2)
    H.HDArrayWrite(A, a, R)
    H.HDArrayWrite(B, b, R)
    out = []
    for bb in (None, None, b2):
        if bb is not None:
            H.HDArrayWrite(B, bb, R)
        H.HDArrayApplyKernel("gemm", R, A, B, C, 1.0, 0.0, ni, nj, nk)
        got = np.zeros((ni, nj), np.float32)
        H.HDArrayRead(C, got, R)
        out.append(got)
    for got, bb in zip(out, (b, b, b2)):
        ref = a.astype(np.float64) @ bb.astype(np.float64)
        assert (np.abs(got - ref) <= 2 * _bf16x3_bound(a, bb, 0 * got, 1.0, 0.0, nk)).all()


# ---------------------------------------------------------------------------------------------
# execution choices must not change results: unfused exchange, autotuned tile shapes, variants
# ---------------------------------------------------------------------------------------------

@pytest.mark.parametrize("env,dtype", [({"HDARRAY_FUSE_EXCHANGE": "0"}, "float"), ({"HDARRAY_AUTOTUNE": "1"}, "float"),
                                       ({"HDARRAY_JACOBI_VARIANT": "0", "HDARRAY_TILE_ROWS": "16"}, "float"),
                                       ({"HDARRAY_JACOBI_VARIANT": "2"}, "float"),
                                       ({"HDARRAY_JACOBI_VARIANT": "2", "HDARRAY_TILE_ROWS": "1"}, "double"),
                                       ({"HDARRAY_JACOBI_VARIANT": "2", "HDARRAY_FUSE_EXCHANGE": "0"}, "float"),
                                       ({"HDARRAY_JACOBI_VARIANT": "3"}, "float"),
                                       ({"HDARRAY_JACOBI_VARIANT": "3", "HDARRAY_BAND2": "3", "HDARRAY_TILE_ROWS": "5"}, "double"),
                                       ({"HDARRAY_JACOBI_VARIANT": "3", "HDARRAY_BAND2": "1", "HDARRAY_TILE_ROWS": "7"}, "bf16"),
                                       ({"HDARRAY_JACOBI_VARIANT": "3", "HDARRAY_FUSE_EXCHANGE": "0"}, "float"),
                                       ({"HDARRAY_JACOBI_VARIANT": "5"}, "float"),
                                       ({"HDARRAY_JACOBI_VARIANT": "5", "HDARRAY_BAND2": "64"}, "float"),
                                       ({"HDARRAY_JACOBI_VARIANT": "5", "HDARRAY_BAND2": "3", "HDARRAY_TILE_ROWS": "5"}, "double"),
                                       ({"HDARRAY_JACOBI_VARIANT": "5", "HDARRAY_BAND2": "1", "HDARRAY_TILE_ROWS": "7"}, "bf16"),
                                       ({"HDARRAY_JACOBI_VARIANT": "5", "HDARRAY_TILE_ROWS": "1"}, "bf16"),
                                       ({"HDARRAY_JACOBI_VARIANT": "5", "HDARRAY_FUSE_EXCHANGE": "0"}, "float")])
def test_jacobi2d_execution_choices(gpu_lib, monkeypatch, env, dtype):
    for k, v in env.items():
        monkeypatch.setenv(k, v)
    dims, P = (260, 530), 6
    x = synthetic.jacobi_field(dims, stream=81, dtype=dtype)
    prog, last = jacobi_prog(dims, P, 7, BLOCK, dtype, True)
    lib, orc, *_ = run_program(prog, P, {"B": x, "A": x}, gpu_lib)
    assert np.array_equal(read_all(lib, last, dims, dtype), orc.arrays[last].G)


def test_batch_flat_variant(gpu_lib, monkeypatch):
    monkeypatch.setenv("HDARRAY_JACOBI_VARIANT", "2")
    test_batch_of_instances(gpu_lib)


def test_batch_packed_variant(gpu_lib, monkeypatch):
    monkeypatch.setenv("HDARRAY_JACOBI_VARIANT", "3")
    monkeypatch.setenv("HDARRAY_TILE_ROWS", "9")
    test_batch_of_instances(gpu_lib)


def test_batch_tma_variant(gpu_lib, monkeypatch):
    """Rows staged by bulk tensor copies: every instance's parts with their own tensor maps, merged
    into one launch."""
    monkeypatch.setenv("HDARRAY_JACOBI_VARIANT", "5")
    monkeypatch.setenv("HDARRAY_TILE_ROWS", "3")
    test_batch_of_instances(gpu_lib)


@pytest.mark.parametrize("dims,P,ptype,dtype,band", [((150, 70), 7, COL, "float", "32"), ((150, 70), 7, COL, "bf16", "32"),
                                                     ((300, 45), 11, COL, "double", "32"), ((64, 900), 9, ROW, "float", "8"),
                                                     ((97, 131), 16, COL, "float", "2")])
@pytest.mark.parametrize("variant", ["3", "5"])
def test_jacobi2d_packed_narrow(gpu_lib, monkeypatch, dims, P, ptype, dtype, band, variant):
    """Packed row streams, and rows staged by bulk tensor copies, on partitions a few elements wide
    or a few rows high."""
    monkeypatch.setenv("HDARRAY_JACOBI_VARIANT", variant)
    monkeypatch.setenv("HDARRAY_BAND2", band)
    monkeypatch.setenv("HDARRAY_TILE_ROWS", "6")
    x = synthetic.jacobi_field(dims, stream=87, dtype=dtype)
    prog, last = jacobi_prog(dims, P, 5, ptype, dtype, True)
    lib, orc, *_ = run_program(prog, P, {"B": x, "A": x}, gpu_lib)
    assert np.array_equal(read_all(lib, last, dims, dtype), orc.arrays[last].G)


@pytest.mark.parametrize("dims,P,ptype,dtype,rows,band", [
    ((700, 300), 5, COL, "float", "40", "16"),    # tiles longer than the ring: later stages read the buffer
    ((2600, 200), 3, COL, "float", "80", "16"),   # middle parts receive 1280 elements a tile: receive first
    ((300, 500), 6, ROW, "bf16", "8", "32"),      # row faces, patched into the first and the last stage
    ((257, 263), 9, BLOCK, "double", "12", "16")])
@pytest.mark.parametrize("late", ["0", "1"])
def test_jacobi2d_tma_late_receive(gpu_lib, monkeypatch, dims, P, ptype, dtype, rows, band, late):
    """Rows staged by bulk tensor copies with the receive before the tile's first copies (late 0) or
    after them, the received values patched into the stages already copied (late 1): every held
    element of every device buffer and the result are the oracle's."""
    monkeypatch.setenv("HDARRAY_JACOBI_VARIANT", "5")
    monkeypatch.setenv("HDARRAY_TILE_ROWS", rows)
    monkeypatch.setenv("HDARRAY_BAND2", band)
    monkeypatch.setenv("HDARRAY_LATE_RECEIVE", late)
    x = synthetic.jacobi_field(dims, stream=89, dtype=dtype)
    prog, last = jacobi_prog(dims, P, 5, ptype, dtype, True)
    lib, orc, *_ = run_program(prog, P, {"B": x, "A": x}, gpu_lib)
    assert np.array_equal(read_all(lib, last, dims, dtype), orc.arrays[last].G)


@pytest.mark.parametrize("variant", ["0", "1", "3", "5"])
@pytest.mark.parametrize("dtype", ["float", "bf16"])
def test_jacobi2d_special_values(gpu_lib, monkeypatch, variant, dtype):
    """Subnormal values and results, infinities, sums that overflow to infinity and signed zeros:
    every kernel form rounds each cell exactly as the oracle's binary32 arithmetic."""
    monkeypatch.setenv("HDARRAY_JACOBI_VARIANT", variant)
    monkeypatch.setenv("HDARRAY_TILE_ROWS", "10")
    dims, P = (150, 270), 6
    x = synthetic.jacobi_field(dims, stream=88, dtype="double")
    x[1:30, :] *= 2.0 ** -130                 # subnormal binary32 and bfloat16 values and results
    x[40:43, 100:104] = np.inf
    x[60, 50:53] = 3.0e38                      # neighbours whose sum overflows
    x[80:90, 30:40] = -0.0                     # all-negative-zero neighbourhoods: -0 * 0.25 = -0
    x[100:110, 200:210] = -x[100:110, 200:210]
    x = synthetic.to_storage(x, dtype)
    prog, last = jacobi_prog(dims, P, 4, BLOCK, dtype, True)
    lib, orc, *_ = run_program(prog, P, {"B": x, "A": x}, gpu_lib)
    got = read_all(lib, last, dims, dtype)
    want = orc.arrays[last].G
    wf = want.astype(np.float32) if dtype == "float" else oracle.bf16_to_f32(want)
    assert np.isinf(wf).any() and ((wf != 0) & (np.abs(wf) < 2.0 ** -126)).any() and np.signbit(wf[wf == 0]).any()
    assert np.array_equal(got.view(np.uint8), want.view(np.uint8))


@pytest.mark.parametrize("env,dtype", [({"HDARRAY_FUSE_EXCHANGE": "0"}, "float"), ({"HDARRAY_AUTOTUNE": "1"}, "float"),
                                       ({"HDARRAY_STENCIL3D_VARIANT": "0"}, "float"), ({"HDARRAY_TILE_Z": "7"}, "float"),
                                       ({"HDARRAY_STENCIL3D_VARIANT": "2"}, "float"),
                                       ({"HDARRAY_STENCIL3D_VARIANT": "2", "HDARRAY_TILE_ROWS": "1"}, "double"),
                                       ({"HDARRAY_STENCIL3D_VARIANT": "2", "HDARRAY_TILE_Z": "5"}, "float"),
                                       ({"HDARRAY_STENCIL3D_VARIANT": "3"}, "float"),
                                       ({"HDARRAY_STENCIL3D_VARIANT": "3", "HDARRAY_TILE_Z": "7"}, "double"),
                                       ({"HDARRAY_STENCIL3D_VARIANT": "3", "HDARRAY_FUSE_EXCHANGE": "0"}, "bf16")])
def test_stencil3d_execution_choices(gpu_lib, monkeypatch, env, dtype):
    for k, v in env.items():
        monkeypatch.setenv(k, v)
    n = 36
    boxes = synthetic.kd_boxes(n, 7, stream=82, min_ext=6, max_ext=36)
    x = synthetic.jacobi_field((n, n, n), stream=83, dtype=dtype)
    prog, last = stencil3d_prog(n, boxes, 5, dtype)
    lib, orc, *_ = run_program(prog, len(boxes), {"B": x}, gpu_lib)
    got = np.zeros((n, n, n), NP[dtype])
    H.HDArrayRead(lib.arrays[last], got, lib.parts["D"])
    assert np.array_equal(got, orc.arrays[last].G)


BAND_SHAPES = [("1", "float", "256"), ("4", "float", "256"), ("16", "float", "256"), ("64", "float", "256"),
               ("3", "bf16", "256"), ("64", "bf16", "256"), ("5", "double", "256"), ("64", "double", "256"),
               ("1", "float", "512"), ("32", "float", "512"), ("512", "float", "512"), ("7", "bf16", "512"),
               ("64", "double", "512")]


@pytest.mark.parametrize("variant", ["1", "3"])
@pytest.mark.parametrize("band,dtype,cta", BAND_SHAPES)
def test_stencil3d_cta_band_shapes(gpu_lib, monkeypatch, band, dtype, cta, variant):
    """The CTA kernels' tiles follow the box: narrow bands with many rows, wide bands with few,
    bands of equal width across a row (the last one narrower), ragged last tiles in y and z, with
    256 or 512 threads; the planes staged by cp.async (variant 1) or by bulk tensor copies of a box
    per plane (variant 3, whose boxes of a part's ragged tiles reach past the buffer and read
    zeros)."""
    monkeypatch.setenv("HDARRAY_STENCIL3D_VARIANT", variant)
    monkeypatch.setenv("HDARRAY_BAND3", band)
    monkeypatch.setenv("HDARRAY_CTA3", cta)
    monkeypatch.setenv("HDARRAY_TILE_Z", "9")
    n = 44
    dims = (n, n, 150)
    boxes = [((0, 0, 0), (20, 44, 3)), ((0, 0, 3), (20, 44, 17)), ((0, 0, 17), (20, 30, 150)),
             ((0, 30, 17), (20, 44, 150)), ((20, 0, 0), (44, 7, 150)), ((20, 7, 0), (44, 44, 61)),
             ((20, 7, 61), (44, 44, 150))]
    work = [(tuple(max(1, v) for v in lo), tuple(min(d - 1, v) for v, d in zip(hi, dims))) for lo, hi in boxes]
    x = synthetic.jacobi_field(dims, stream=84, dtype=dtype)
    prog = [("create", "B", dtype, dims), ("create", "A", dtype, dims),
            ("manual", "D", dims, boxes), ("manual", "W", dims, work), ("write", "B", "D")]
    a, b = "B", "A"
    for _ in range(4):
        prog.append(("apply", "stencil3d", "W", [a, b]))
        a, b = b, a
    lib, orc, *_ = run_program(prog, len(boxes), {"B": x}, gpu_lib)
    got = np.zeros(dims, NP[dtype])
    H.HDArrayRead(lib.arrays[a], got, lib.parts["D"])
    assert np.array_equal(got.view(np.uint8), orc.arrays[a].G.view(np.uint8))


@pytest.mark.parametrize("variant", ["0", "1", "2", "3"])
def test_stencil3d_special_values(gpu_lib, monkeypatch, variant):
    """Sums outside the fast division's range -- subnormal and tiny values, infinities, signed
    zeros -- are divided exactly as IEEE division does (bit-exact against the oracle's s / 6)."""
    monkeypatch.setenv("HDARRAY_STENCIL3D_VARIANT", variant)
    n = 30
    boxes = synthetic.kd_boxes(n, 5, stream=85, min_ext=6, max_ext=30)
    x = synthetic.jacobi_field((n, n, n), stream=86, dtype="float")
    x[:, :10, :] *= np.float32(2.0 ** -120)   # sums near 2^-118: below the fast method's range
    x[:, 10:13, :] *= np.float32(2.0 ** -135)  # subnormal values and results
    x[3:6, 20, 7:9] = np.inf
    x[12, 25, 3] = np.float32(3.0e38)          # large finite values next to each other
    x[12, 25, 4] = np.float32(3.0e38)
    x[20:25, 14:17, 2:5] = np.float32(-0.0)     # all-negative-zero neighbourhoods: -0 / 6 = -0
    prog, last = stencil3d_prog(n, boxes, 3, "float")
    lib, orc, *_ = run_program(prog, len(boxes), {"B": x}, gpu_lib)
    got = np.zeros((n, n, n), np.float32)
    H.HDArrayRead(lib.arrays[last], got, lib.parts["D"])
    want = orc.arrays[last].G
    assert np.isinf(want).any() and (np.abs(want[(want != 0) & np.isfinite(want)]) < 2.0 ** -100).any()
    assert np.array_equal(np.isnan(got), np.isnan(want))
    ok = ~np.isnan(want)
    assert np.array_equal(got[ok].view(np.uint32), want[ok].view(np.uint32))


# ---------------------------------------------------------------------------------------------
# 2-D convolution (Sec. 5: eight neighbours and the centre, weights as scalars)
# ---------------------------------------------------------------------------------------------

def conv_prog(dims, P, ptype, dtype, w):
    prog = [("create", "X", dtype, dims), ("create", "Y", dtype, dims),
            ("part", "D", ptype, dims, (0, 0), dims, P),
            ("part", "W", ptype, dims, (1, 1), tuple(n - 1 for n in dims), P),
            ("write", "X", "D"), ("write", "Y", "D")]
    # X -> Y, then Y -> X (moves Y's halo rows, columns and corners), then X -> Y with X unchanged
    for src, dst in (("X", "Y"), ("Y", "X"), ("X", "Y"), ("X", "Y")):
        prog.append(("apply", "conv2d", "W", [src, dst], list(w)))
    return prog


CONV_CASES = [((130, 301), 4, BLOCK, "float"), ((97, 131), 3, ROW, "double"), ((140, 270), 5, COL, "bf16"),
              ((70, 600), 2, ROW, "bf16"), ((150, 70), 7, COL, "float"), ((259, 515), 6, BLOCK, "double")]


@pytest.mark.parametrize("dims,P,ptype,dtype", CONV_CASES)
@pytest.mark.parametrize("mode", [H.HDARRAY_MODE_FUSED, H.HDARRAY_MODE_PLAIN])
@pytest.mark.parametrize("variant", ["3", "5"])
def test_conv2d_parity(gpu_lib, monkeypatch, dims, P, ptype, dtype, mode, variant):
    """Every storage type and partition shape, fused and plain, with the packed-stream kernel and
    with rows staged by bulk tensor copies."""
    monkeypatch.setenv("HDARRAY_JACOBI_VARIANT", variant)
    monkeypatch.setenv("HDARRAY_TILE_ROWS", "5")
    x = synthetic.jacobi_field(dims, stream=94, dtype=dtype)
    w = synthetic.normal(9, stream=95) * 0.3
    lib, orc, *_ = run_program(conv_prog(dims, P, ptype, dtype, w), P, {"X": x, "Y": x}, gpu_lib, mode=mode)
    for name in ("X", "Y"):
        assert np.array_equal(read_all(lib, name, dims, dtype), orc.arrays[name].G)


@pytest.mark.parametrize("env", [{"HDARRAY_BAND2": "1", "HDARRAY_TILE_ROWS": "3"}, {"HDARRAY_BAND2": "3"},
                                 {"HDARRAY_FUSE_EXCHANGE": "0"}, {"HDARRAY_AUTOTUNE": "1"},
                                 {"HDARRAY_BAND2": "32", "HDARRAY_TILE_ROWS": "64"},
                                 {"HDARRAY_JACOBI_VARIANT": "5", "HDARRAY_BAND2": "1", "HDARRAY_TILE_ROWS": "1"},
                                 {"HDARRAY_JACOBI_VARIANT": "5", "HDARRAY_BAND2": "64"},
                                 {"HDARRAY_JACOBI_VARIANT": "5", "HDARRAY_FUSE_EXCHANGE": "0"}])
def test_conv2d_execution_choices(gpu_lib, monkeypatch, env):
    for k, v in env.items():
        monkeypatch.setenv(k, v)
    dims, P = (203, 389), 6
    x = synthetic.jacobi_field(dims, stream=96, dtype="float")
    w = synthetic.normal(9, stream=97)
    lib, orc, *_ = run_program(conv_prog(dims, P, BLOCK, "float", w), P, {"X": x, "Y": x}, gpu_lib)
    for name in ("X", "Y"):
        assert np.array_equal(read_all(lib, name, dims, "float"), orc.arrays[name].G)


@pytest.mark.parametrize("rows,variant", [(None, None), ("16", None), ("16", "5")])
def test_conv2d_full_size_8192_block16(gpu_lib, rows, variant, monkeypatch):
    """The convolution workload at full size (8192^2 binary32, BLOCK 4 x 4) in a graph; outputs
    sampled at partition corners and edges and at random, each recomputed by the oracle from its
    3 x 3 neighbourhood; default tile rows, the autotuned 16, and rows staged by TMA."""
    if rows:
        monkeypatch.setenv("HDARRAY_TILE_ROWS", rows)
    if variant:
        monkeypatch.setenv("HDARRAY_JACOBI_VARIANT", variant)
    N, P = 8192, 16
    x = synthetic.jacobi_field((N, N), stream=98, dtype="float")
    w = synthetic.normal(9, stream=99)
    gpu_lib(P)
    X = H.HDArrayCreate("X", "float", None, N, N)
    Y = H.HDArrayCreate("Y", "float", None, N, N)
    D = H.HDArrayPartition(H.BLOCK, (N, N), (0, 0), (N, N), P)
    Wp = H.HDArrayPartition(H.BLOCK, (N, N), (1, 1), (N - 1, N - 1), P)
    H.HDArrayWrite(X, x, D)
    H.HDArrayApplyKernel("conv2d", Wp, X, Y, *w)
    H.HDArrayGraphBegin()
    H.HDArrayApplyKernel("conv2d", Wp, X, Y, *w)
    gid = H.HDArrayGraphEnd()
    H.HDArrayGraphLaunch(gid, 3)
    got = np.zeros((N, N), np.float32)
    H.HDArrayRead(Y, got, D)
    rng = np.random.default_rng(11)
    samples = [tuple(int(v) for v in rng.integers(1, N - 1, 2)) for _ in range(40)]
    for b in (2047, 2048, 2049, 4095, 4096, 6143, 6144):  # BLOCK 4 x 4 boundaries of the work region
        samples += [(b, 1), (1, b), (b, b), (b, N - 2), (N - 2, b)]
    samples += [(1, 1), (N - 2, N - 2), (1, N - 2), (N - 2, 1)]
    L = oracle.lib()
    wv = np.ascontiguousarray(w, dtype=np.float64)
    for (i, j) in samples:
        win = np.ascontiguousarray(x[i - 1:i + 2, j - 1:j + 2])
        out = np.zeros((3, 3), np.float32)
        work = np.zeros((3, 3), np.uint8)
        work[1, 1] = 1
        assert L.orc_conv2d(1, 3, 3, win.ctypes.data, out.ctypes.data, work.ctypes.data, wv.ctypes.data) == 0
        assert got[i, j].view(np.uint32) == out[1, 1].view(np.uint32), (i, j)


# ---------------------------------------------------------------------------------------------
# 2MM on row and column blocks (Sec. 5.1): the same products, different exchanges
# ---------------------------------------------------------------------------------------------

def two_mm_prog(n, P, ptype, iters, dtype):
    prog = [("create", x, dtype, (n, n)) for x in "ABCDE"]
    prog += [("part", "Q", ptype, (n, n), (0, 0), (n, n), P)]
    prog += [("write", x, "Q") for x in "ABCDE"]
    for _ in range(iters):
        prog.append(("apply", "gemm", "Q", ["A", "B", "D"], (1.0, 0.0, n, n, n)))
        prog.append(("apply", "gemm", "Q", ["C", "D", "E"], (1.0, 0.0, n, n, n)))
    return prog


@pytest.mark.parametrize("ptype", [ROW, COL, BLOCK])
@pytest.mark.parametrize("dtype,n,P", [("double", 96, 4), ("float", 320, 4), ("float", 512, 2), ("float", 200, 6)])
def test_2mm_parity(gpu_lib, ptype, dtype, n, P):
    vals = {x: synthetic.to_storage(synthetic.normal(n * n, stream=100 + i).reshape(n, n), dtype)
            for i, x in enumerate("ABCDE")}
    lib, orc, *_ = run_program(two_mm_prog(n, P, ptype, 2, dtype), P, vals, gpu_lib, check_buffers=False)
    got = {x: read_all(lib, x, (n, n), dtype, "Q").astype(np.float64) for x in "DE"}
    A, B, C = (vals[x].astype(np.float64) for x in "ABC")
    if dtype == "double":
        for x in "DE":
            ref = orc.arrays[x].G
            assert np.abs(got[x] - ref).max() <= 1e-12 * np.abs(ref).max()
    else:
        # each product within the bf16x3 bound of its own (binary32) operands as stored on the GPU
        z = np.zeros((n, n), np.float32)
        assert (np.abs(got["D"] - A @ B) <= 2 * _bf16x3_bound(vals["A"], vals["B"], z, 1.0, 0.0, n)).all()
        D32 = got["D"].astype(np.float32)
        assert (np.abs(got["E"] - C @ D32.astype(np.float64)) <= 2 * _bf16x3_bound(vals["C"], D32, z, 1.0, 0.0, n)).all()


# ---------------------------------------------------------------------------------------------
# covariance (Sec. 5.1): triangular product with absolute / trapezoid sections, symmetric copy
# ---------------------------------------------------------------------------------------------

@pytest.mark.parametrize("balanced,correlation", [(False, False), (True, False), (False, True)])
@pytest.mark.parametrize("dtype,n,m,P", [("double", 70, 96, 4), ("float", 300, 384, 4), ("float", 130, 200, 3)])
def test_covariance_parity(gpu_lib, balanced, correlation, dtype, n, m, P):
    from cov_program import cov_prog
    prog, rows = cov_prog(n, m, P, dtype=dtype, balanced=balanced, correlation=correlation)
    x = synthetic.to_storage(synthetic.normal(n * m, stream=110).reshape(n, m) + 0.5, dtype)
    lib, orc, *_ = run_program(prog, P, {"X": x}, gpu_lib, check_buffers=False)
    M = read_all(lib, "M", (1, m), dtype, "PM").astype(np.float64)
    Xc = read_all(lib, "Xc", (n, m), dtype, "DX")
    C = read_all(lib, "C", (m, m), dtype, "PC")
    # means: binary64 sums in another order (each within (n - 1) 2^-53 sum|x| of the exact sum),
    # then rounded to the storage type (one unit in the last place of the stored mean)
    Mo = orc.arrays["M"].G.astype(np.float64)
    sums = 2 * (n + 1) * 2.0 ** -53 * np.abs(x.astype(np.float64)).sum(axis=0) / n
    ulp = 0.0 if dtype == "double" else 2.0 ** -23
    assert (np.abs(M - Mo) <= sums + ulp * np.abs(Mo) + 1e-300).all()
    # centring is one subtraction in the storage precision of the device's own means
    assert np.array_equal(Xc, (x - M.astype(x.dtype)).astype(x.dtype))
    # the symmetric copy is exact
    assert np.array_equal(C, C.T)
    alpha = 1.0 / (n - 1)
    if correlation:  # unit-norm columns: S within the summation bound, the scaling one division
        S = read_all(lib, "S", (1, m), dtype, "PM").astype(np.float64)
        Xc64 = Xc.astype(np.float64)
        Sref = np.sqrt((Xc64 ** 2).sum(axis=0))
        assert (np.abs(S - Sref) <= (n + 2) * 2.0 ** -53 * Sref + (0 if dtype == "double" else 2.0 ** -23 * Sref)).all()
        Xs = read_all(lib, "Xs", (n, m), dtype, "DX")
        assert np.array_equal(Xs, (Xc / S.astype(Xc.dtype)).astype(Xc.dtype))
        Xc, alpha = Xs, 1.0
    # the product: within the rounding bound of the arithmetic used, against the device's own input
    X64 = Xc.astype(np.float64)
    ref = alpha * X64.T @ X64
    mag = alpha * np.abs(X64).T @ np.abs(X64)
    if dtype == "double":
        bound = 2 * (n + 2) * 2.0 ** -53 * mag + 1e-300
    else:
        bound = 2 * _bf16x3_bound(Xc.T.copy(), Xc, np.zeros((m, m), np.float32), alpha, 0.0, n)
    assert (np.abs(C.astype(np.float64) - ref) <= bound).all()
    # and the oracle's matrix agrees with numpy's
    want = np.corrcoef(x.astype(np.float64), rowvar=False) if correlation else np.cov(x.astype(np.float64), rowvar=False)
    assert np.abs(orc.arrays["C"].G.astype(np.float64) - want).max() <= (1e-12 if dtype == "double" else 1e-4) * np.abs(want).max()


@pytest.mark.parametrize("balanced", [False, True])
def test_covariance_bf16x6(gpu_lib, balanced):
    """The triangular product (transposed A, upper-triangle output, 128-column tiles) in the bf16x6
    form: within its bound and within 1e-5 of |X^T||X| componentwise; messages as the oracle's."""
    from cov_program import cov_prog
    n, m, P = 300, 384, 4
    prog, rows = cov_prog(n, m, P, dtype="float", balanced=balanced)
    x = synthetic.to_storage(synthetic.normal(n * m, stream=111).reshape(n, m) + 0.5, "float")
    lib, orc, *_ = run_program(prog, P, {"X": x}, gpu_lib, check_buffers=False,
                               setup=lambda: H.HDArraySetGemmSplit(H.HDARRAY_GEMM_BF16X6))
    Xc = read_all(lib, "Xc", (n, m), "float", "DX")
    C = read_all(lib, "C", (m, m), "float", "PC")
    assert np.array_equal(C, C.T)
    alpha = 1.0 / (n - 1)
    X64 = Xc.astype(np.float64)
    err = np.abs(C.astype(np.float64) - alpha * X64.T @ X64)
    bound, mag = _bf16x6_bound(Xc.T.copy(), Xc, np.zeros((m, m), np.float32), alpha, 0.0, n)
    assert (err <= bound).all(), float((err / bound).max())
    assert (err <= 1e-5 * mag).all(), float((err / mag).max())


def test_gemm_split_setting(gpu_lib):
    """HDArraySetGemmSplit accepts the two forms only, and not inside a batch."""
    gpu_lib(2)
    with pytest.raises(H.HDArrayError):
        H.HDArraySetGemmSplit(4)
    H.HDArrayBatchBegin()
    with pytest.raises(H.HDArrayError):
        H.HDArraySetGemmSplit(H.HDARRAY_GEMM_BF16X6)
    H.HDArrayBatchEnd()
    H.HDArraySetGemmSplit(H.HDARRAY_GEMM_BF16X6)
    H.HDArraySetGemmSplit(H.HDARRAY_GEMM_BF16X3)


# ---------------------------------------------------------------------------------------------
# user kernels (HDArrayRegisterKernel) and a caller-supplied allocator (HDArraySetAllocator)
# ---------------------------------------------------------------------------------------------

@pytest.mark.parametrize("dtype", ["float", "double"])
@pytest.mark.parametrize("ptype,P", [(BLOCK, 6), (COL, 5), (ROW, 3)])
@pytest.mark.parametrize("mode", [H.HDARRAY_MODE_FUSED, H.HDARRAY_MODE_PLAIN])
def test_user_kernel_parity(gpu_lib, dtype, ptype, P, mode):
    """A user kernel (torch on views of the library's buffers) behind the library's exchange:
    messages and values equal the oracle's, including a kernel with scalars, in a graph replay."""
    torch = pytest.importorskip("torch")
    import user_kernels
    user_kernels.register_oracle()
    np_t = NP[dtype]

    def setup():
        H.HDArrayRegisterKernel("max4", 2, 0, 1, user_kernels.max4_launcher(torch, np_t))
        H.HDArraySetOffsetUse("max4", 0, user_kernels.J4)
        H.HDArraySetOffsetDef("max4", 1, [(0, 0)])
        H.HDArrayRegisterKernel("axpb", 2, 2, 1, user_kernels.axpb_launcher(torch, np_t))
        H.HDArraySetOffsetUse("axpb", 0, [(0, 0)])
        H.HDArraySetOffsetDef("axpb", 1, [(0, 0)])

    dims = (130, 117)
    x = synthetic.to_storage(synthetic.normal(dims[0] * dims[1], stream=120).reshape(dims), dtype)
    prog = [("create", "B", dtype, dims), ("create", "A", dtype, dims),
            ("part", "D", ptype, dims, (0, 0), dims, P), ("part", "W", ptype, dims, (1, 1), (dims[0] - 1, dims[1] - 1), P),
            ("write", "B", "D"), ("write", "A", "D")]
    for i in range(4):
        src, dst = ("B", "A") if i % 2 == 0 else ("A", "B")
        prog.append(("apply", "max4", "W", [src, dst]))
        prog.append(("apply", "axpb", "W", [dst, dst == "A" and "B" or "A"], (0.5, -0.25)))
        prog.append(("apply", "max4", "W", [dst == "A" and "B" or "A", dst]))
    lib, orc, *_ = run_program(prog, P, {"B": x, "A": x}, gpu_lib, mode=mode, setup=setup)
    for name in ("A", "B"):
        assert np.array_equal(read_all(lib, name, dims, dtype), orc.arrays[name].G)


def test_user_kernel_error_code(gpu_lib):
    gpu_lib(2)
    H.HDArrayRegisterKernel("fails", 2, 0, 1, lambda work, scal, stream: -4)
    H.HDArraySetOffsetUse("fails", 0, [(0, 0)])
    H.HDArraySetOffsetDef("fails", 1, [(0, 0)])
    X = H.HDArrayCreate("X", "float", None, 16, 16)
    Y = H.HDArrayCreate("Y", "float", None, 16, 16)
    Pp = H.HDArrayPartition(H.ROW, (16, 16), (0, 0), (16, 16), 2)
    with pytest.raises(H.HDArrayError) as e:
        H.HDArrayApplyKernel("fails", Pp, X, Y)
    assert e.value.code == -4


def test_caller_allocator(gpu_lib):
    """Array buffers and tables from torch's caching allocator: results unchanged, every
    allocation and release went through it."""
    torch = pytest.importorskip("torch")
    calls = {"alloc": 0, "free": 0}
    live = set()

    def alloc(n):
        p = torch.cuda.caching_allocator_alloc(n)
        calls["alloc"] += 1
        live.add(p)
        return p

    def free(p):
        calls["free"] += 1
        live.discard(p)
        torch.cuda.caching_allocator_delete(p)

    H.HDArraySetAllocator(alloc, free)
    try:
        dims, P = (150, 201), 4
        x = synthetic.jacobi_field(dims, stream=121, dtype="float")
        prog, last = jacobi_prog(dims, P, 6, BLOCK, "float", True)
        lib, orc, *_ = run_program(prog, P, {"B": x, "A": x}, gpu_lib)
        assert np.array_equal(read_all(lib, last, dims, "float"), orc.arrays[last].G)
        assert calls["alloc"] > 0
        H.HDArrayExit()
        assert calls["free"] == calls["alloc"] and not live
    finally:
        H.HDArraySetAllocator(None, None)


# ---------------------------------------------------------------------------------------------
# full sizes of the batch and triangular-GEMM workloads, in the launch form bench.py times,
# checked on sampled outputs the oracle computes one by one
# ---------------------------------------------------------------------------------------------

def test_full_size_batch_512_instances(gpu_lib):
    """512 instances (sides log-uniform 64..2048, 2-16 ROW/COL parts, FP32), merged into one
    launch per iteration inside a graph, 200 iterations; samples in 24 instances (partition
    boundaries, corners, random) against the oracle's light cone."""
    insts = synthetic.jacobi_instances(512, stream=5)
    ndev = max(p for _, _, p, _ in insts)
    gpu_lib(ndev)
    arrs, xs = [], []
    for i, (r, c, P, kind) in enumerate(insts):
        t = ROW if kind == "ROW" else COL
        x = synthetic.jacobi_field((r, c), stream=1000 + i, dtype="float")
        B = H.HDArrayCreate("B", "float", None, r, c)
        A = H.HDArrayCreate("A", "float", None, r, c)
        D = H.HDArrayPartition(t, (r, c), (0, 0), (r, c), P)
        W = H.HDArrayPartition(t, (r, c), (1, 1), (r - 1, c - 1), P)
        H.HDArrayWrite(B, x, D)
        arrs.append((B, A, D, W))
        xs.append(x)

    def iteration(flip):
        H.HDArrayBatchBegin()
        for B, A, D, W in arrs:
            H.HDArrayApplyKernel("jacobi2d", W, *((A, B) if flip else (B, A)))
        H.HDArrayBatchEnd()

    T = 200
    for _ in range(2):
        iteration(False)
        iteration(True)
    H.HDArrayGraphBegin()
    iteration(False)
    iteration(True)
    gid = H.HDArrayGraphEnd()  # recording also ran its two iterations
    H.HDArrayGraphLaunch(gid, (T - 6) // 2)
    rng = np.random.default_rng(17)
    for i in rng.choice(len(insts), 24, replace=False):
        r, c, P, kind = insts[i]
        B, A, D, W = arrs[i]
        got = np.zeros((r, c), np.float32)
        H.HDArrayRead(B, got, D)
        bx = oracle.partition_boxes(ROW if kind == "ROW" else COL, P, (r, c), (1, 1), (r - 1, c - 1))
        samples = [tuple(int(v) for v in rng.integers(1, (r - 1, c - 1))) for _ in range(2)]
        for lo, hi in bx[:3]:  # partition edges: the exchanged halo matters here
            samples.append((lo[0], lo[1]))
            samples.append((hi[0] - 1, hi[1] - 1))
        want = light_cone(xs[i], 1, samples, T)
        gotv = np.array([got[s] for s in samples])
        assert np.array_equal(gotv, want), "instance %d" % i


@pytest.mark.parametrize("dtype,split", [("double", 0), ("float", 2), ("float", 3)])
def test_full_size_trmm_8192x4096(gpu_lib, dtype, split):
    """tril(A) 8192^2 x B 8192x4096 on 8 row blocks with trapezoid use sections (binary64 on the
    DFMA pipe, binary32 on the tensor cores): sampled entries against the oracle's exact binary64
    entries (FP64 within 1e-12 relative to |A||B|, bf16x3 within its bound)."""
    n, m, P = 8192, 4096, 8
    a, b = synthetic.tri_gemm_inputs(n, m, stream=4, dtype=dtype)
    gpu_lib(P)
    if split == 3:
        H.HDArraySetGemmSplit(H.HDARRAY_GEMM_BF16X6)
    A = H.HDArrayCreate("A", dtype, None, n, n)
    B = H.HDArrayCreate("B", dtype, None, n, m)
    C = H.HDArrayCreate("C", dtype, None, n, m)
    R = H.HDArrayPartition(H.ROW, (n, m), (0, 0), (n, m), P)
    RA = H.HDArrayPartition(H.ROW, (n, n), (0, 0), (n, n), P)
    rows = [n * p // P for p in range(P + 1)]
    for p in range(P):
        r0, r1 = rows[p], rows[p + 1]
        H.HDArraySetTrapezoidUse("trmm", R, A, p, (r0, 0, r0, r0, r1 - 1, 0, r1 - 1, r1 - 1))
    H.HDArrayWrite(A, a, RA)
    H.HDArrayWrite(B, b, R)
    H.HDArrayApplyKernel("trmm", R, A, B, C, 1.0, 0.0)
    got = np.zeros((n, m), NP[dtype])
    H.HDArrayRead(C, got, R)
    rng = np.random.default_rng(23)
    ij = [(int(rng.integers(0, n)), int(rng.integers(0, m))) for _ in range(200)]
    ij += [(r, 0) for r in rows[1:-1]] + [(r - 1, m - 1) for r in rows[1:]] + [(0, 0), (n - 1, m - 1)]
    ij = np.ascontiguousarray(np.array(ij, np.int64))
    A64, B64 = np.tril(a.astype(np.float64)), b.astype(np.float64)
    want = np.zeros(len(ij))
    oracle.lib().orc_gemm_entries(m, n, 1.0, 0.0, A64.ctypes.data, B64.ctypes.data, None, len(ij),
                                  ij.ctypes.data, want.ctypes.data)
    gotv = np.array([got[i, j] for i, j in ij], np.float64)
    mag = np.array([np.abs(A64[i, :i + 1]) @ np.abs(B64[:i + 1, j]) for i, j in ij])
    k = np.array([i + 1 for i, _ in ij])
    if dtype == "double":
        assert (np.abs(gotv - want) <= 1e-12 * mag).all()
    elif split == 2:
        assert (np.abs(gotv - want) <= 2 * (3 * 2.0 ** -16 + (k + 2) * 2.0 ** -24) * mag).all()
    else:  # bf16x6: its bound, and binary32 accuracy (1e-5 of |A||B| componentwise)
        assert (np.abs(gotv - want) <= (4 + 6 * k + 2) * 2.0 ** -24 * mag).all()
        assert (np.abs(gotv - want) <= 1e-5 * mag).all()
