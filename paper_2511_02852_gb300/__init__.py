"""GB300-native (sm_103a) hybrid wave-particle / FFT ocean height-field
synthesis of arXiv 2511.02852 behind a C ABI (``include/scwp.h``).

``scwp`` is the ctypes binding (same call names as the C ABI);
``workloads`` describes the seeded synthetic scenes; ``_build`` compiles the
CUDA library in-tree.
"""
__all__ = ["scwp", "workloads"]
