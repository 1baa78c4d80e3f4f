"""GB300-native Boltzmann--ES-BGK flux-reconstruction stage (arXiv 2312.06567).

The compute path is the C-ABI library ``libbgk.so`` built from ``csrc/`` for
sm_103a; :mod:`.bgk` is its thin ctypes binding.  Importing this package does
not load the library; the first call into :mod:`.bgk` does, and raises if it
is missing.
"""
