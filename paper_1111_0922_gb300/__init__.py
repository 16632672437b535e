"""GB300-native D3Q19 lattice Boltzmann propagation-step library.

The compute path is the C-ABI shared library ``liblbm.so`` built from
``csrc/`` (hand-written sm_103a CUDA kernels).  ``lbm`` is its thin ctypes
binding; importing this package does not load the library, so the seeded
input generators in ``inputs`` stay usable on machines without a GPU.
"""
__all__ = ["inputs", "model"]
