"""GB300-native Tucker (HOSVD) approximation of Matern covariance tensors.

The compute path is the CUDA library ``libtucker_matern.so`` (sm_103a) behind
the C-ABI declared in ``include/tucker_matern.h``; ``binding`` marshals
arguments to it.  Importing this package does not load the library; the first
call into ``binding`` does, and raises if it is missing.
"""
__all__ = ["binding", "workloads"]
