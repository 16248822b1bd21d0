"""GB300-native SIMUS RF hot path: Green's-term generation, scatterer reduction and
transmit contraction in hand-written sm_103a CUDA behind a C-ABI (``include/simus.h``).

Importing the package loads nothing; ``paper_2102_02738_gb300.simus`` loads the CUDA
library and raises if it is missing.
"""
__all__ = ["simus", "phantoms"]
