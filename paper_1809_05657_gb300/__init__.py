"""GB300 HDArray: arrays split over logical devices, with automatic section exchange.

The library (libhdarray.so, built from csrc/ by build.py) implements the hot path of
HDArrayApplyKernel on one GB300: def/use section intersection (Eq. 1-4 of the paper), the
section moves between logical-device buffers, and the kernels.  hdarray.py binds its C ABI.
"""
from . import hdarray  # noqa: F401
from .hdarray import *  # noqa: F401,F403
