"""GB300-native phase-field lattice Boltzmann solver for droplets on wetting
walls (arXiv 2312.00369): CUDA kernels for sm_103a behind the C ABI of
include/pflbm.h, with a thin ctypes binding.

Importing the package loads nothing; ``paper_2312_00369_gb300.pflbm`` loads
``libpflbm.so`` on first use and raises if it is missing.
"""
__all__ = ["pflbm", "workloads", "build"]
