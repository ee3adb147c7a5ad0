"""GB300-native NeDF composition renderer (arXiv 2308.04669).

Submodules:
  scenegen  seeded synthetic scenes (inputs only)
  native    ctypes binding of the C-ABI library libnedf_compose.so (loaded on import; raises if
            the library has not been built)
  build     compiles the CUDA library for sm_103a
"""
