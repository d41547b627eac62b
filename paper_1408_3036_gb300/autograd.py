"""s = <phi|eps~^-1(0)|phi> as a differentiable function of the local potential.

``EpsInvQuad.apply(vloc, phi, L, ecut, n_occ, k, prec)`` returns s for the
cell of edge L whose local potential is ``vloc`` (N^3 values on the grid) and
back-propagates ds/dV_loc(r) (not in the paper: the adjoint of third-order
perturbation theory, see gw_grad_vloc in include/gw.h).

Forward: one context for this V_loc (gw_setup), its lowest n_occ states (the
input preparation of groundstate.lowest_states), k Lanczos steps on eps~(0)
from phi with the basis kept (gw_lanczos), T^-1 (gw_epsinv_elements),
s = |phi|^2 (T^-1)_11.  The Lanczos basis, alpha and beta are the checkpoint
saved for backward (k N^3 doubles).

Backward: gw_grad_vloc_basis on the same context: u = |phi| Q T^-1 e_1, the
Sternheimer solves for the first-order orbitals and the adjoint solves, which
are recomputed there and never held between the passes.

Marshalling only: every step runs in libgw's kernels.  phi is not
differentiated (its gradient is returned as None).
"""
from __future__ import annotations

import torch

from . import GW_FP64, Cell, gw_epsinv_elements, gw_grad_vloc_basis, gw_lanczos
from .groundstate import lowest_states


class EpsInvQuad(torch.autograd.Function):
    @staticmethod
    def forward(ctx, vloc, phi, L, ecut, n_occ, k, prec=GW_FP64):
        if vloc.dtype != torch.float64 or phi.dtype != torch.float64:
            raise ValueError("vloc and phi must be float64")
        ng = vloc.numel()
        N = round(ng ** (1.0 / 3.0))
        if N ** 3 != ng or phi.numel() != ng:
            raise ValueError("vloc and phi must hold N^3 values")
        dev = phi.device
        if dev.type != "cuda":
            raise ValueError("phi must be a CUDA tensor")
        cell = Cell(L, N, ecut, vloc.detach().reshape(-1).cpu().numpy())
        eps, psi, res = lowest_states(cell, n_occ, tol=1e-11)
        if res > 1e-9:
            cell.close()
            raise RuntimeError(f"ground state did not converge (residual {res:.2e})")
        cell.set_occupied(psi[:n_occ], eps[:n_occ])
        phi_c = phi.detach().reshape(-1).contiguous()
        alpha = torch.empty(k, dtype=torch.float64, device=dev)
        beta = torch.empty(max(k - 1, 1), dtype=torch.float64, device=dev)
        Q = torch.empty((k, ng), dtype=torch.float64, device=dev)
        gw_lanczos(cell.ctx, phi_c, k, 0.0, alpha, beta, Q, prec)
        Ti = torch.empty((k, k), dtype=torch.float64, device=dev)
        gw_epsinv_elements(cell.ctx, alpha, beta, k, Ti)
        wgt = float(L) ** 3 / ng
        s = (phi_c * phi_c).sum() * wgt * Ti[0, 0]
        ctx.save_for_backward(phi_c, Q, alpha, beta)
        ctx.cell, ctx.k, ctx.prec, ctx.shape = cell, k, prec, vloc.shape
        return s

    @staticmethod
    def backward(ctx, grad_s):
        phi_c, Q, alpha, beta = ctx.saved_tensors
        dev = phi_c.device
        grad = torch.empty_like(phi_c)
        s = torch.empty(1, dtype=torch.float64, device=dev)
        gw_grad_vloc_basis(ctx.cell.ctx, phi_c, Q, alpha, beta, ctx.k, s, grad, ctx.prec)
        ctx.cell.close()
        return (grad_s * grad).reshape(ctx.shape), None, None, None, None, None, None


def checkpoint_bytes(N, k):
    """Device bytes of the checkpoint kept between forward and backward: the
    Lanczos basis (k N^3 doubles) and alpha, beta."""
    return 8 * (k * N ** 3 + 2 * k)


def orbital_bytes(N, npw, n_occ):
    """Device bytes of what the checkpoint avoids keeping: the first-order
    orbitals dpsi_v and adjoint solutions lambda_v in the sphere (complex FP64)
    and dpsi_v on the grid."""
    return 16 * (2 * n_occ * npw + n_occ * N ** 3)
