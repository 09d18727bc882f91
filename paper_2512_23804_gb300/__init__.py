"""GB300-native stochastic Galerkin KKT solver for PDE-constrained optimisation
under uncertain diffusion coefficients (hierarchical Gauss-Seidel preconditioned
MINRES, steady and all-at-once time-dependent).

The computation lives in the CUDA library libsgoc.so behind the C ABI of
include/sgoc.h; `abi` binds it with ctypes and `SGProblem` manages device
memory and streams through PyTorch.
"""
from . import abi
from .problem import SGProblem, SGServer, solve_batch

__all__ = ["abi", "SGProblem", "SGServer", "solve_batch"]
