"""GB300-native TEBD two-site bond update with reduced-rank randomized SVD.

The compute path is a C-ABI shared library of hand-written sm_103a CUDA
kernels (``libtebd_gb300.so``); :mod:`.binding` is its thin ctypes binding.
Importing the package does not load the library, so that the pure-NumPy input
generators in :mod:`.inputs` stay usable on machines without a GPU; every
compute call goes through the binding, which raises if the library or a CUDA
device is missing.
"""
__all__ = ["binding", "inputs", "build"]
