"""Failure detection without faulting the GPU: a device-side wait made to run out (a limit of
zero polls) is reported as HDARRAY_ERR_TIMEOUT and leaves the context usable; allocation
failures injected through the allocator hook are reported as errors; host-side misuse is
rejected before anything is launched."""

import numpy as np
import pytest

import synthetic
from paper_1809_05657_gb300 import hdarray as H

TIMEOUT, NOMEM, INVAL = -5, -2, -1


@pytest.fixture
def gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from __graft_entry__ import build_library
    build_library()
    torch.cuda.init()
    yield torch
    H.HDArrayExit()
    H.HDArraySetAllocator(None, None)


def _gemm_f32(n, P):
    a = synthetic.to_storage(synthetic.normal(n * n, stream=130).reshape(n, n), "float")
    b = synthetic.to_storage(synthetic.normal(n * n, stream=131).reshape(n, n), "float")
    A, B, C = (H.HDArrayCreate(x, "float", None, n, n) for x in "ABC")
    R = H.HDArrayPartition(H.ROW, (n, n), (0, 0), (n, n), P)
    H.HDArrayWrite(A, a, R)
    H.HDArrayWrite(B, b, R)
    H.HDArrayWrite(C, np.zeros((n, n), np.float32), R)
    return A, B, C, R, a, b


@pytest.mark.gpu
def test_gemm_pipeline_wait_timeout_is_reported(gpu, monkeypatch):
    monkeypatch.setenv("HDARRAY_SPIN_LIMIT", "0")  # every pipeline wait gives up at once
    H.HDArrayInit(ndev=2)
    A, B, C, R, a, b = _gemm_f32(256, 2)
    H.HDArrayApplyKernel("gemm", R, A, B, C, 1.0, 0.0, 256, 256, 256)
    with pytest.raises(H.HDArrayError) as e:
        H.HDArraySync()
    assert e.value.code == TIMEOUT
    H.HDArraySync()  # reported once; the context is still usable
    H.HDArrayExit()
    monkeypatch.delenv("HDARRAY_SPIN_LIMIT")
    H.HDArrayInit(ndev=2)
    A, B, C, R, a, b = _gemm_f32(256, 2)
    H.HDArrayApplyKernel("gemm", R, A, B, C, 1.0, 0.0, 256, 256, 256)
    got = np.zeros((256, 256), np.float32)
    H.HDArrayRead(C, got, R)
    ref = a.astype(np.float64) @ b.astype(np.float64)
    assert np.abs(got - ref).max() <= 1e-4 * np.abs(ref).max()


@pytest.mark.gpu
def test_allocation_failure_is_reported(gpu):
    H.HDArraySetAllocator(lambda n: 0, lambda p: None)  # every allocation fails
    H.HDArrayInit(ndev=2)
    X = H.HDArrayCreate("X", "float", None, 64, 64)
    D = H.HDArrayPartition(H.ROW, (64, 64), (0, 0), (64, 64), 2)
    with pytest.raises(H.HDArrayError) as e:
        H.HDArrayWrite(X, np.zeros((64, 64), np.float32), D)
    assert e.value.code == NOMEM


@pytest.mark.gpu
def test_misaligned_allocation_is_rejected(gpu):
    torch = gpu
    held = []

    def alloc(n):
        p = torch.cuda.caching_allocator_alloc(n + 512)
        held.append(p)
        return p + 16  # 16-byte aligned only

    H.HDArraySetAllocator(alloc, lambda p: torch.cuda.caching_allocator_delete(p - 16))
    H.HDArrayInit(ndev=2)
    X = H.HDArrayCreate("X", "float", None, 64, 64)
    D = H.HDArrayPartition(H.ROW, (64, 64), (0, 0), (64, 64), 2)
    with pytest.raises(H.HDArrayError) as e:
        H.HDArrayWrite(X, np.zeros((64, 64), np.float32), D)
    assert e.value.code == INVAL


@pytest.mark.gpu
def test_stencil3d_bulk_copy_wait_timeout_is_reported(gpu, monkeypatch):
    """The 3-D kernel whose planes arrive by bulk tensor copies: with a limit of zero polls every
    wait on a plane gives up, the tiles compute nothing, the copies already issued are waited for,
    and the call reports HDARRAY_ERR_TIMEOUT once; then the context computes correctly."""
    import oracle
    monkeypatch.setenv("HDARRAY_STENCIL3D_VARIANT", "3")
    n = 34
    boxes = synthetic.kd_boxes(n, 5, stream=87, min_ext=6, max_ext=34)
    work = [(tuple(max(1, v) for v in lo), tuple(min(n - 1, v) for v in hi)) for lo, hi in boxes]
    x = synthetic.jacobi_field((n, n, n), stream=88, dtype="float")

    def program():
        B = H.HDArrayCreate("B", "float", None, n, n, n)
        A = H.HDArrayCreate("A", "float", None, n, n, n)
        D = H.HDArrayPartitionManual((n, n, n), boxes)
        W = H.HDArrayPartitionManual((n, n, n), work)
        H.HDArrayWrite(B, x, D)
        H.HDArrayApplyKernel("stencil3d", W, B, A)
        return A, D

    monkeypatch.setenv("HDARRAY_SPIN_LIMIT", "0")
    H.HDArrayInit(ndev=len(boxes))
    program()
    with pytest.raises(H.HDArrayError) as e:
        H.HDArraySync()
    assert e.value.code == TIMEOUT
    H.HDArraySync()  # reported once
    H.HDArrayExit()
    monkeypatch.delenv("HDARRAY_SPIN_LIMIT")
    H.HDArrayInit(ndev=len(boxes))
    A, D = program()
    got = np.zeros((n, n, n), np.float32)
    H.HDArrayRead(A, got, D)
    o = oracle.Oracle(len(boxes))
    ob, oa = o.create("B", "float", (n, n, n)), o.create("A", "float", (n, n, n))
    od = o.partition_manual(boxes)
    o.write(ob, x, od)
    o.apply("stencil3d", o.partition_manual(work), [ob, oa])
    assert np.array_equal(got, oa.G)


@pytest.mark.gpu
def test_jacobi2d_bulk_copy_wait_timeout_is_reported(gpu, monkeypatch):
    """The 2-D kernel whose rows arrive by bulk tensor copies: with a limit of zero polls every wait
    on a stage gives up, the tiles compute nothing, the copies already issued are waited for, and
    the call reports HDARRAY_ERR_TIMEOUT once; then the context computes correctly."""
    import oracle
    monkeypatch.setenv("HDARRAY_JACOBI_VARIANT", "5")
    dims, P = (200, 330), 6
    x = synthetic.jacobi_field(dims, stream=89, dtype="float")

    def program():
        B = H.HDArrayCreate("B", "float", None, *dims)
        A = H.HDArrayCreate("A", "float", None, *dims)
        D = H.HDArrayPartition(H.BLOCK, dims, (0, 0), dims, P)
        W = H.HDArrayPartition(H.BLOCK, dims, (1, 1), (dims[0] - 1, dims[1] - 1), P)
        H.HDArrayWrite(B, x, D)
        H.HDArrayApplyKernel("jacobi2d", W, B, A)
        return A, D

    monkeypatch.setenv("HDARRAY_SPIN_LIMIT", "0")
    H.HDArrayInit(ndev=P)
    program()
    with pytest.raises(H.HDArrayError) as e:
        H.HDArraySync()
    assert e.value.code == TIMEOUT
    H.HDArraySync()  # reported once
    H.HDArrayExit()
    monkeypatch.delenv("HDARRAY_SPIN_LIMIT")
    H.HDArrayInit(ndev=P)
    A, D = program()
    got = np.zeros(dims, np.float32)
    H.HDArrayRead(A, got, D)
    o = oracle.Oracle(P)
    ob, oa = o.create("B", "float", dims), o.create("A", "float", dims)
    od = o.partition(oracle.BLOCK, dims, (0, 0), dims)
    o.write(ob, x, od)
    o.apply("jacobi2d", o.partition(oracle.BLOCK, dims, (1, 1), (dims[0] - 1, dims[1] - 1)), [ob, oa])
    assert np.array_equal(got, oa.G)
