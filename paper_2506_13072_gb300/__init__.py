"""GB300-native library for the fluctuating lattice Boltzmann method for
Oldroyd-B fluids (arXiv 2506.13072).

The compute path is the CUDA library built from ``csrc/`` (C ABI in
``include/fvlb.h``); ``fvlb`` is its Python binding and ``workloads`` holds the
seeded synthetic problems shaped like the paper's test flows.  Importing the
binding requires the built library: ``paper_2506_13072_gb300.build.build()``.
"""
__all__ = ["fvlb", "workloads", "build"]
