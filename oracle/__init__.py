"""CPU oracle for the hierarchical Hough transform (test infrastructure only).

Only the tests, the smoke check and the benchmark's CPU-baseline leg may import
this package.  It loads `hht_oracle.c` (plain C, compiled with gcc on first
use) through ctypes and shares no code with the CUDA library.
"""
from .oracle import (  # noqa: F401
    build,
    loaded_path,
    detect,
    count_region,
    getcode,
    scaled_F,
    fht_votes,
    frame_side,
    sobel,
    edges,
    detect_split,
    detect_subtrees,
    detect_removal,
    lines,
    line_parameters,
    centroid_parameters,
    LINE_DTYPE,
    OracleResult,
    STAT_TESTED,
    STAT_PASSED,
    STAT_VOTES,
    STAT_TESTS,
)
