"""gx: GB300-native breadth-first exploration of networks of synchronising LTSs.

Submodules:
  gx      -- ctypes binding of the C ABI in include/gx.h (the CUDA library)
  inputs  -- seeded synthetic networks and key sequences
  build   -- in-tree build of the CUDA library for sm_103a

Importing the package loads nothing; the CUDA library is loaded on the first
call into ``gx``.
"""
