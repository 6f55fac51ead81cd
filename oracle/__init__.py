"""Plain CPU oracle for the HDArray hot path (test infrastructure only).

Only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline leg may import this package.
See hdarray_oracle.c for what it computes and oracle.py for the program driver.
"""
from .oracle import *  # noqa: F401,F403
from .oracle import Oracle, KERNELS, lib, partition_boxes, gemm_entries, f32_to_bf16, bf16_to_f32  # noqa: F401
