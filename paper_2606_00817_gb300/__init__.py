"""GB300-native batched Directed Distance Field queries.

Submodules:
  ddf     -- ctypes binding of the C-ABI library ``libddf.so`` (the product path)
  inputs  -- seeded synthetic rays, scenes and weights
  build   -- compiles the CUDA library for sm_103a
The package imports nothing heavy at import time.
"""
__all__ = ["ddf", "inputs", "build"]
