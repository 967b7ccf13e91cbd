"""GB300-native builder and query engine for pointerless level-wise wavelet trees.

The CUDA library (``libwt.so``, built from ``csrc/``) is reached through the
C ABI declared in ``include/wt.h``; :mod:`.wt` is the thin ctypes binding and
:mod:`.inputs` the seeded synthetic sequence generator.  Importing the package
loads nothing; the binding loads the library on first use and raises if it is
missing.
"""
