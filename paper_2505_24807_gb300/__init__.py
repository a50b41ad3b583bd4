"""GB300-native semiempirical CIS / TDHF excited states (libxs).

The compute path is the C-ABI library ``libxs.so`` built from ``csrc/`` for
sm_103a; ``xs`` is its thin ctypes binding.  Importing this package does not
load the library; ``paper_2505_24807_gb300.xs`` does, and fails loudly when it
has not been built.
"""
