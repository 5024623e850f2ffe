"""GB300-native face-staggered susceptibility artifact correction (SAC).

The compute path lives in the C-ABI library ``libsac.so`` (hand-written CUDA
for sm_103a, built from ``csrc/``); ``paper_1607_00531_gb300.sac`` is its thin
ctypes binding.  Importing this package loads nothing.
"""
__all__ = ["sac", "phantoms"]
