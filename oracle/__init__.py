"""FP64 CPU oracle of the DMSGM block-grid step (arXiv:1702.05156, Sec. 2.2-2.4)
and of the preprocessing filters (Sec. 2.1).

TEST INFRASTRUCTURE ONLY: tests, the smoke check and the benchmark's CPU
baseline leg use it to check and time the CUDA library.  The product package
never imports it.
"""
from .oracle import (  # noqa: F401
    DIAG,
    OracleState,
    build_oracle,
    gauss_weights,
    oracle_run,
    oracle_step,
    prefilter,
    state_from_arrays,
)
