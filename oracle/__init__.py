"""CPU oracle for the sample Tukey depth count -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  It wraps ``tukey_oracle.c`` (plain C,
exact integer arithmetic) through ctypes and shares no code with the CUDA
library.
"""
from .oracle import (  # noqa: F401
    build,
    depth,
    depth_many,
    depth_range,
    subset_min,
    bivariate_closed,
    rank,
    adia,
    critical,
    ADIA_STATS,
    OracleError,
)
