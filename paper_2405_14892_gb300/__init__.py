"""GB300-native SOV estimation of high-dimensional multivariate normal probabilities.

The compute path is the C-ABI library ``libmvn.so`` (CUDA kernels for sm_103a, declared in
``include/mvn.h``); the Python functions in ``paper_2405_14892_gb300.mvn`` are thin ctypes
bindings with the same names.  Importing this package does not load the library; the first call
of a binding does, and fails loudly when it is missing.
"""
