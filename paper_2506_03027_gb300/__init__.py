"""GB300-native asynchronous compressible flow solver (arXiv 2506.03027 hot path).

The compute lives in a C-ABI CUDA library (``libcfs.so``, built by ``build.py``); ``cfs`` is its
thin ctypes binding and ``inputs`` holds the seeded synthetic workloads.  Importing the package
loads nothing: ``cfs.load()`` opens the library and fails loudly when it is missing.
"""
__all__ = ["cfs", "inputs"]
