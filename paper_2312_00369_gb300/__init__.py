"""GB300-native phase-field lattice Boltzmann solver for droplets on wetting
walls (arXiv 2312.00369), in 2D (D2Q9) and 3D (D3Q19 / D3Q7): CUDA kernels
for sm_103a behind the C ABI of include/pflbm.h, with a thin ctypes binding,
batched and served solves.

Importing the package loads nothing; ``paper_2312_00369_gb300.pflbm`` loads
``libpflbm.so`` on first use and raises if it is missing.
"""
__all__ = ["pflbm", "workloads", "build"]
