"""GB300-native cascadic multigrid Fiedler-vector solver (Gandhi 2015, Alg. 3).

The compute path is the CUDA library built from ``csrc/`` (C-ABI in
``include/fiedler.h``); ``fiedler`` is its thin ctypes binding and ``inputs``
the seeded synthetic graph generators.  Importing the package loads nothing;
the library is loaded (and must exist) on first use of ``fiedler``.
"""
__all__ = ["fiedler", "inputs", "build"]
