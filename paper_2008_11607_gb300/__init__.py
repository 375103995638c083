"""GB300-native REXII time step for the linear rotating shallow-water equations.

The compute path lives in ``csrc/`` (CUDA for sm_103a behind a C ABI declared
in ``include/rexi.h``); ``rexi`` is the thin ctypes binding with the same entry
points.  ``inputs`` holds the seeded synthetic workloads.  Importing this
package does not load the CUDA library; ``rexi.load()`` does, and fails loudly
when it is missing.
"""
__all__ = ["inputs", "rexi"]
