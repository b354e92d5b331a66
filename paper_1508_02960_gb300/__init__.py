"""GB300-native fused D3Q19 lattice Boltzmann hot path for periodic sphere packs
(Fattahi et al., arXiv:1508.02960).

The compute path lives in the CUDA library built from ``csrc/`` (``liblbm_gb300.so``);
``capi`` is its ctypes binding.  Importing the package does not load the library; the
first call into ``capi`` does, and raises if the library is missing.
"""
__all__ = ["capi", "inputs"]
