"""GB300 (sm_103a) library for the total-Lagrangian vectorial lattice
Boltzmann method for finite-strain hyperelastic dynamics (Feng & Chu).

The compute path is the CUDA library built from csrc/ (C ABI in
include/lbm.h); ``paper_2605_26677_gb300.lbm`` is its Python binding. There is
no CPU fallback: importing ``lbm`` fails if the library has not been built.
"""
__all__ = ["build", "lbm"]
