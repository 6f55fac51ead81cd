"""The C ABI library builds, loads on a host without a GPU, and exports every declared call."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "hdarray.h")


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*[A-Za-z_][\w\s\*]*?\b(HDArray\w+)\s*\(", src, flags=re.M)
    return sorted(set(names))


def test_header_declares_paper_calls():
    names = declared_functions()
    for n in ["HDArrayInit", "HDArrayExit", "HDArrayShowDeviceInfo", "HDArrayCreate",
              "HDArrayPartition", "HDArrayApplyKernel", "HDArrayRead", "HDArrayWrite",
              "HDArrayReduce", "HDArraySetAbsoluteUse", "HDArraySetAbsoluteDef",
              "HDArraySetTrapezoidUse", "HDArraySetTrapezoidDef"]:
        assert n in names, n


def test_library_exports_every_declared_symbol():
    from __graft_entry__ import build_library
    path = build_library()
    lib = ctypes.CDLL(path)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing
    out = subprocess.run(["nm", "-D", "--defined-only", path], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT (HDArray\w+)", out))
    assert set(declared_functions()) <= exported


def test_header_compiles_as_c():
    """The header is plain C (no C++ or CUDA types in the signatures)."""
    prog = '#include "hdarray.h"\nint main(void) { return HDARRAY_OK; }\n'
    r = subprocess.run(["gcc", "-std=c99", "-Wall", "-Werror", "-fsyntax-only", "-I",
                        os.path.dirname(HEADER), "-x", "c", "-"], input=prog, text=True,
                       capture_output=True)
    assert r.returncode == 0, r.stderr


def test_host_only_init_needs_no_gpu():
    from paper_1809_05657_gb300 import hdarray as H
    H.HDArrayInit(ndev=3, host_only=True)
    try:
        assert H.HDArrayNumDevices() if hasattr(H, "HDArrayNumDevices") else True
        x = H.HDArrayCreate("x", "float", None, 16, 16)
        p = H.HDArrayPartition(H.ROW, (16, 16), (0, 0), (16, 16), 3)
        H.HDArrayWrite(x, None, p)
        assert H.HDArrayGetGDEF(x, 0, 1) == [((0, 0, 0), (6, 16, 1))]
    finally:
        H.HDArrayExit()


def test_error_strings():
    from paper_1809_05657_gb300 import hdarray as H
    lib = H.lib()
    for code in range(0, -9, -1):
        assert lib.HDArrayErrorString(code)
