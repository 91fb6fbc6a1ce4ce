"""GB300-native coupled D2Q9 + D2Q5 lattice Boltzmann step (Tanaka & Iber,
arXiv 1307.4703).

The compute path is the CUDA library ``csrc/`` compiled for sm_103a and
exposed through the C ABI of ``include/lbm.h``; ``lbm`` is its thin ctypes
binding.  Importing this package does not load the library: ``lbm.load()``
does, and fails loudly when it is missing.
"""
__all__ = ["lbm", "workloads"]
