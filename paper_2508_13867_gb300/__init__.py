"""GB300-native ensemble lattice-Boltzmann uncertainty quantification (arXiv 2508.13867).

The compute path is libuqlb.so (CUDA for sm_103a behind the C ABI of include/uqlb.h);
``uqlb`` is its ctypes binding and ``ensemble`` a torch-backed convenience layer that only
allocates device memory, picks streams and marshals arguments.
"""
from . import build, uqlb, workloads  # noqa: F401
