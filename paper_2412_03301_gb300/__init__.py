"""GB300-native BioVSS++ query path (arXiv 2412.03301).

The compute runs in hand-written CUDA kernels for sm_103a behind the C ABI
declared in ``include/bvss.h``; ``paper_2412_03301_gb300.bvss`` is the thin
Python binding with the same names.  Importing this package loads nothing;
the binding loads the shared library on first use and raises if it is
missing.
"""
