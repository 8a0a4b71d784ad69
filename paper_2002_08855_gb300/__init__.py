"""GB300-native IB-LBM hot path for particle-laden flows.

The compute path is ``libibmlbm.so`` (hand-written CUDA for sm_103a behind a
C ABI declared in ``include/ibmlbm.h``); ``binding`` marshals arguments to it
through ctypes and uses PyTorch only for device memory and streams.  Importing
this package loads nothing: the library is opened on first use and a missing
library raises instead of falling back to any other implementation.
"""

__all__ = ["binding", "inputs"]
