"""FP64 CPU oracle of the DMSGM block-grid step (arXiv:1702.05156, Sec. 2.2-2.4),
of the preprocessing filters (Sec. 2.1) and of the motion-estimation front
end that produces the homography (Sec. 2.4, Sec. 3.1.3).

TEST INFRASTRUCTURE ONLY: tests, the smoke check and the benchmark's CPU
baseline leg use it to check and time the CUDA library.  The product package
never imports it.
"""
from .oracle import (  # noqa: F401
    DIAG,
    HOMOG_DEFAULTS,
    corners,
    estimate_homography,
    hypothesis,
    inliers,
    pyr_down,
    ransac,
    ransac_counts,
    refit,
    sample4,
    score_map,
    tensor_map,
    set_threads,
    splitmix64,
    track,
    OracleState,
    build_oracle,
    gauss_weights,
    oracle_run,
    oracle_step,
    prefilter,
    state_from_arrays,
)
