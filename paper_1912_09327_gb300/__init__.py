"""GB300-native LBMTau1: the fused moments-only D2Q9 stream-and-collide step
of Matyka & Dzikowski, "Memory-efficient Lattice Boltzmann Method for low
Reynolds number flows" (arXiv:1912.09327), as sm_103a CUDA behind a C ABI.

Importing the package loads nothing; ``paper_1912_09327_gb300.binding``
loads the shared library and fails loudly when it is missing.
"""

__all__ = ["binding", "workloads"]
