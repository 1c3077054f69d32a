"""torch.autograd wrapper of the adjoint FMG solve (no counterpart in the paper).

`L2Functional.apply(f_L, k, mesh, in_S, params, g_L)` returns J(u) = u^T M_S u, the squared L2 norm of
the level-L solution u over the macro cells flagged in `in_S`, where u solves the HHG system with
source f_L (level-L layout, one value per interface copy) and per-cell coefficients k.

Gradients come from one adjoint solve in the library (hhg_adjoint_l2), run in forward only when
f_L or k requires a gradient; otherwise forward evaluates J from the solution alone.  The forward
solution is kept by the mesh, not stored by autograd.

dJ/df_L is the derivative with respect to every entry of f_L: the library builds b_L = sum_T M_T f_T
from each cell's own copy of an interface node, so copy p of cell T gets (M_T lambda)_p.  An
upstream op that spreads nodal values to the copies (f_L = f_nodes[idx]) therefore sums the copies'
shares into the nodal derivative (M_L lambda)_p.
"""

from __future__ import annotations

import numpy as np
import torch

from .hhg import Mesh, solve_params


class L2Functional(torch.autograd.Function):
    @staticmethod
    def forward(ctx, f_L, k, mesh: Mesh, in_S, params, g_L):
        if not f_L.is_cuda:
            raise ValueError("f_L must be a CUDA tensor in the mesh's level-L layout")
        kk = k.detach().to("cpu", torch.float64).numpy()
        mesh.set_coefficient(kk)
        f = f_L.detach().to(torch.float64).contiguous()
        g = g_L.detach().to(device=f.device, dtype=torch.float64).contiguous()
        mesh.set_data(f, g)
        u = torch.empty_like(f)
        mesh.solve(params, out=u)
        mask = np.asarray(in_S, dtype=np.uint8)
        ctx.k_device = k.device
        ctx.k_dtype = k.dtype
        if ctx.needs_input_grad[0] or ctx.needs_input_grad[1]:
            grad_f = torch.empty_like(f)
            J, _, grad_k = mesh.adjoint_l2(mask, params=params, grad_f=grad_f)
            ctx.save_for_backward(grad_f, torch.from_numpy(grad_k))
        else:
            # no gradient wanted: J = sum over the flagged cells of u^T M_T u, from the solution alone
            sq = torch.empty(mesh.n_cells, dtype=torch.float64, device=f.device)
            mesh.cell_mass_norms_noalloc(u, None, sq)
            mesh.synchronize()
            J = float(sq.cpu().numpy()[mask.astype(bool)].sum())
        return torch.tensor(J, dtype=torch.float64, device=f.device)

    @staticmethod
    def backward(ctx, gJ):
        grad_f, grad_k = ctx.saved_tensors
        gf = gJ * grad_f
        gk = (gJ.to("cpu") * grad_k).to(device=ctx.k_device, dtype=ctx.k_dtype)
        return gf, gk, None, None, None, None


def l2_functional(f_L, k, mesh, in_S, g_L=None, params=None):
    """J(u(f_L, k)) = u^T M_S u with gradients through torch.autograd."""
    if params is None:
        params = solve_params(nu=2, pre=2, post=1, n_extra=40)
    if g_L is None:
        g_L = torch.zeros_like(f_L)
    return L2Functional.apply(f_L, k, mesh, in_S, params, g_L)
