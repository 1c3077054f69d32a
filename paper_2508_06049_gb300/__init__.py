"""GB300-native full multigrid on hierarchical hybrid grids with the FMG error estimator.

The compute path is the CUDA library libhhg.so (C ABI in include/hhg.h); this package only
binds it.  See hhg.py for the binding and autograd.py for the torch.autograd wrapper of the
adjoint solve.
"""

from .hhg import (  # noqa: F401
    HHGError, Mesh, RG2D, RG3D, SolveParams, lattice_selfcheck, lib, mark, solve_params,
)
