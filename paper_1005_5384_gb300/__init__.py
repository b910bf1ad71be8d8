"""GB300-native grouped Barnes-Hut tree-code force calculation (Gaburov, Bedorf &
Portegies Zwart 2010, "Gravitational tree-code on graphics processing units").

The compute path is a C-ABI shared library (host FP64 octree build + sm_103a CUDA
walk/evaluation kernels); ``paper_1005_5384_gb300.octgrav`` is its thin ctypes
binding. Importing the package itself loads nothing.
"""
__all__ = ["octgrav", "workloads"]
