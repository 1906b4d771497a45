"""Compressed full-state quantum circuit simulation on one GB300 (sm_103a).

The compute path is the C-ABI library ``libqcsim.so`` built from ``csrc/``; the
``qcsim`` module is its ctypes binding.  ``circuits`` holds the seeded input
generators.  Importing this package loads nothing: the library is loaded on first use.
"""
__all__ = ["circuits", "qcsim"]
