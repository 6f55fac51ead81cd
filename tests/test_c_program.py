"""The C ABI used from C: a Listing-2-style host program (variadic paper calls) is compiled with
gcc against include/hdarray.h and libhdarray.so; on a GPU its result equals the oracle's."""

import os
import subprocess

import numpy as np
import pytest

from oracle import Oracle, ROW

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "tests", "c_listing2_jacobi.c")
PKG = os.path.join(ROOT, "paper_1809_05657_gb300")


def compile_program(tmp_path):
    from __graft_entry__ import build_library
    build_library()
    exe = str(tmp_path / "c_listing2_jacobi")
    cmd = ["gcc", "-O2", "-std=c11", "-Wall", "-I", os.path.join(ROOT, "include"), SRC, "-L", PKG, "-lhdarray",
           "-Wl,-rpath," + PKG, "-o", exe]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    return exe


def test_c_program_builds_against_the_abi(tmp_path):
    assert os.path.exists(compile_program(tmp_path))


@pytest.mark.gpu
def test_c_program_matches_oracle(tmp_path):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    exe = compile_program(tmp_path)
    n, iters, P = 96, 7, 3
    dpath = tmp_path / "devices"
    dpath.write_text("%d\n" % P)
    out = tmp_path / "u.bin"
    r = subprocess.run([exe, str(dpath), str(n), str(iters), str(out)], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stderr
    got = np.fromfile(out, np.float64).reshape(n, n)

    u = np.zeros((n, n))
    i, j = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    u[1:-1, 1:-1] = (((i * 31 + j * 17) % 101) / 101.0)[1:-1, 1:-1]
    o = Oracle(P)
    data = o.partition(ROW, (n, n), (0, 0), (n, n))
    work = o.partition(ROW, (n, n), (1, 1), (n - 1, n - 1))
    B = o.create("B", "double", (n, n))
    A = o.create("A", "double", (n, n))
    o.write(B, u, data)
    o.write(A, u, data)
    for _ in range(iters):
        o.apply("jacobi2d", work, [B, A])
        o.apply("copy", work, [A, B])
    assert np.array_equal(got, B.G)
    assert abs(float(r.stdout.strip()) - B.G[1:-1, 1:-1].sum()) <= 1e-12 * B.G[1:-1, 1:-1].sum()
