"""GB300-native FP64 WENO-ZN solver (Shen, Zhang, Li & Peng, arXiv 2004.07954).

The compute path lives in libwenozn.so (hand-written sm_103a CUDA behind a C ABI, declared
in include/wenozn.h); `wenozn` is its thin ctypes binding and `inputs` builds seeded
synthetic initial conditions.  Importing the package loads nothing: the library is loaded
on the first call into `wenozn`.
"""
__all__ = ["wenozn", "inputs", "build"]
