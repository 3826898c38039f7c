"""GENESIS Milne-Eddington GA Stokes inversion for GB300 (sm_103a).

The computation lives in libgenesis.so (include/genesis.h); ``api`` marshals
CUDA tensors into it.  Import ``paper_1208_0302_gb300.api`` for the calls.
"""
__all__ = ["api", "build"]
