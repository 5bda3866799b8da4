"""GB300-native clover Wilson-Dirac operator, Schwarz-preconditioned
mixed-precision FGCR solver and fermion force (arXiv:1109.4279).

The compute path is libqcdgb.so (hand-written CUDA for sm_103a) behind the C
ABI declared in include/qcdgb.h; ``binding`` marshals torch tensors into it.
``synth`` generates seeded synthetic inputs.  Importing the package does not
load the CUDA library; the binding does, and fails loudly if it is missing.
"""
__all__ = ["binding", "synth"]
