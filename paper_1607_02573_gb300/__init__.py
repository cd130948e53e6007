"""GB300-native microwave-imaging solver: edge-element Maxwell solves with
batched ORAS-preconditioned FGMRES, S-parameters, misfit and adjoint gradient.

The computation lives in the CUDA library libmwi.so (C ABI in include/mwi.h);
``mwi`` is its ctypes binding and ``autograd`` exposes the misfit as a
torch.autograd.Function.
"""

__all__ = ["mwi"]
