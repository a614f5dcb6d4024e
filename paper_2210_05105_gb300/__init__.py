"""GB300-native randomized sparse CP decomposition (CP-ARLS-LEV, STS-CP).

The compute path is the CUDA library ``libcpd`` behind the C ABI declared in
``include/cpd.h``; :mod:`.cpd` is the thin ctypes binding over it.  Importing
this package does not load the library; :func:`cpd.lib` does, and raises if it
is missing.
"""
