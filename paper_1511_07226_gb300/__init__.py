"""GB300-native pipelined flexible Krylov solvers (PIPEFCG, PIPEGCR, PIPEFGMRES).

The compute path is the C-ABI library ``libpfk.so`` (hand-written CUDA for
sm_103a, declared in ``include/pfk.h``); ``pfk`` is its thin ctypes binding.
Importing this package does not load the library: ``pfk.load()`` does, and
fails loudly if it has not been built.
"""
