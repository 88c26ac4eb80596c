"""GB300-native adaptive randomized TT-rounding with Khatri-Rao-product sketches.

The compute lives in libttround.so (CUDA for sm_103a, C ABI in include/ttround.h); the
``binding`` submodule is its ctypes binding.  Importing the package does not load the
library; the first call does, and fails loudly if the library has not been built
(``__graft_entry__.build()``).
"""
