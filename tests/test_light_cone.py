"""The light-cone helpers that the full-size GPU tests use against whole oracle runs (CPU)."""
import numpy as np

import oracle
import synthetic
from harness import light_cone, light_cone3


def _full_2d(x, T):
    n0, n1 = x.shape
    B, A = x.copy(), x.copy()
    work = np.zeros(x.shape, np.uint8)
    work[1:-1, 1:-1] = 1
    for _ in range(T):
        assert oracle.lib().orc_jacobi2d(1, n0, n1, B.ctypes.data, A.ctypes.data, work.ctypes.data) == 0
        A, B = B, A
    return B


def test_light_cone_2d_matches_whole_run():
    """Windows clipped by the array and windows covering it all (T beyond both sides)."""
    x = synthetic.jacobi_field((37, 53), stream=77, dtype="float")
    x0 = x.copy()
    samples = [(1, 1), (1, 20), (18, 26), (35, 51), (20, 1)]
    for T in (3, 12, 60):
        got = light_cone(x, 1, samples, T)
        full = _full_2d(x, T)
        assert np.array_equal(got, np.array([full[s] for s in samples])), T
        assert np.array_equal(x, x0)


def test_light_cone_3d_matches_whole_run():
    x = synthetic.jacobi_field((14, 17, 19), stream=78, dtype="float")
    x0 = x.copy()
    samples = [(1, 1, 1), (7, 8, 9), (12, 15, 17)]
    for T in (2, 5, 30):
        B, A = x.copy(), x.copy()
        work = np.zeros(x.shape, np.uint8)
        work[1:-1, 1:-1, 1:-1] = 1
        for _ in range(T):
            assert oracle.lib().orc_stencil3d(1, *x.shape, B.ctypes.data, A.ctypes.data, work.ctypes.data) == 0
            A, B = B, A
        got = light_cone3(x, 1, samples, T)
        assert np.array_equal(got, np.array([B[s] for s in samples])), T
        assert np.array_equal(x, x0)
