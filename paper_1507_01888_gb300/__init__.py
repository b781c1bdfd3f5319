"""GB300-native separated Gaussian-sum operator apply on multiwavelet trees.

The compute lives in libmra.so (CUDA for sm_103a, C ABI in include/mra.h);
``paper_1507_01888_gb300.mra`` is its ctypes binding.  Importing this package
does not load the library; ``mra.load()`` (or any call) does, and fails loudly
if it cannot.
"""
