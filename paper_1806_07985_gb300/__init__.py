"""GB300-native NNCP-HALS with dimension-tree MTTKRP (arXiv:1806.07985).

The compute path is the C-ABI library built from ``csrc/`` (CUDA for sm_103a);
``nncp`` is its thin ctypes binding.  ``synth`` holds the seeded input
generators.  Importing this package does not load the library; the binding
loads it on first use and raises if it is missing.
"""

__all__ = ["nncp", "synth"]
