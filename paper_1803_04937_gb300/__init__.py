"""GB300-native D3Q19 lattice Boltzmann step with the improved equilibrium of
Bauer & Ruede (arXiv:1803.04937).

The compiled library ``liblbm_gb300.so`` (CUDA, sm_103a) is loaded on first use
by :mod:`paper_1803_04937_gb300.lbm`; importing this package alone loads nothing.
"""
__all__ = ["inputs", "lbm", "adjoint"]
