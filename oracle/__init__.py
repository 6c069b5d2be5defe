"""FP64 CPU oracle of the rectangular central-moment LBM (arXiv 2103.02119).

TEST INFRASTRUCTURE ONLY: the test suite, the smoke check and the benchmark's
CPU-baseline / reference arm may import this package; the product path
(``paper_2103_02119_gb300``) never does.

The numerics live in ``rclbm_oracle.c`` (plain C, literal matrix form of the
paper's algorithm).  This module builds it with gcc and wraps it with ctypes.
"""
from .rclbm_oracle import (  # noqa: F401
    Oracle,
    OracleParams,
    build,
    central_moments,
    collide_cell,
    feq,
    lib,
    matrices,
)
