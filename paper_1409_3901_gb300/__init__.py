"""Exact sample Tukey depth on GB300 (sm_103a).

The product is the C-ABI library ``libtukeydepth.so`` built from ``csrc/``;
``paper_1409_3901_gb300.tukey`` is its thin ctypes binding.  Importing the
package itself loads nothing; ``workloads`` holds the seeded input
generators.
"""
__all__ = ["tukey", "workloads"]
