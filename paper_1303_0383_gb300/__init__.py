"""GB300-native local approximate Gaussian-process prediction (Gramacy & Apley,
arXiv:1303.0383): CUDA kernels for sm_103a behind the C ABI of include/lagp.h, with a
thin ctypes binding in :mod:`paper_1303_0383_gb300.lagp`.

Importing the package loads nothing; ``paper_1303_0383_gb300.lagp.load()`` (called by
every binding function) builds or loads liblagp.so and raises if it cannot.
"""
__all__ = ["lagp", "inputs", "build"]
