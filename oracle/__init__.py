"""CPU FP64 oracle for the HHG full-multigrid solver and error estimator.

TEST INFRASTRUCTURE ONLY.  Only the test suite, ``__graft_entry__.smoke()`` and
the CPU-baseline leg of ``bench.py`` may import this package.  The product
path (the CUDA library and its Python binding) never imports, links or calls
it, and shares no code with it.

The oracle is deliberately plain and slow: it refines every macro element
recursively (red refinement in 2D, Bey's rule in 3D) with integer barycentric
node keys, assembles global sparse matrices element by element, and runs the
paper's Alg. 4 (FMG + ErrorEstimate) step by step with a direct coarse solve.
"""

from .hhg_oracle import (  # noqa: F401
    Hierarchy, fmg, vcycle, smooth, estimate, mark_top_fraction,
    theorem41_constants, corollary_dgamma_bounds, RG2D, adjoint_gradients,
    local_mass_sq, l2_error_sq,
)
