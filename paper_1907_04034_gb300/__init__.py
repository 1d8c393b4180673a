"""GB300-native EDAC weakly-compressible SPH with an inlet and the hybrid
non-reflecting outlet (arXiv 1907.04034).

The compute path is the C-ABI library ``libedac.so`` built from ``csrc/`` (CUDA
for sm_103a); ``binding`` wraps it with ctypes and uses PyTorch only for device
memory and streams.  ``cases`` holds the seeded problem generators.  Importing
the package does not load the CUDA library; ``binding.load()`` does, and fails
loudly when it is missing.
"""
__all__ = ["cases", "binding"]
