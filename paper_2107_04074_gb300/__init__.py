"""GB300-native spherical k-means (arXiv 2107.04074): the Lloyd iteration with
cosine Elkan / Hamerly bounds, as a CUDA library with a C ABI (include/skm.h).

Submodules: ``skm`` (the ctypes binding) and ``build`` (compiles the library
with nvcc).
"""
