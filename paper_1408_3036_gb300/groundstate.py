"""Lowest eigenpairs of H = |G|^2/2 + V_loc on the GPU (input preparation).

The method takes the DFT occupied states as input (Sec. Results: ABINIT
ground states converged to squared residual < 1e-12 Ha^2).  For synthetic
cells this module produces them: block LOBPCG whose H applications are the
library's CUDA H-apply (gw_apply_h, FP64); the small Rayleigh-Ritz problems use
torch on the device.  Not part of the dielectric hot path.
"""
from __future__ import annotations

import math

import numpy as np

from . import GW_FP64, gw_apply_h


def lowest_states(cell, n, tol=1e-10, max_iter=400, extra=None, seed=0, verbose=False):
    """Return (eps[n + 1], psi[n, npw] complex128 numpy, max residual).

    The (n+1)-th eigenvalue is included so that the caller can check the gap
    above the highest occupied state."""
    import torch
    dev = torch.device("cuda")
    npw = cell.npw
    m = n + 1 + (extra if extra is not None else max(4, n // 4))
    miller = torch.tensor(cell.sphere(), dtype=torch.float64, device=dev)
    kin = 0.5 * (2 * math.pi / cell.L) ** 2 * (miller ** 2).sum(1)
    prec = 1.0 / (kin + 1.0)
    g = torch.Generator(device="cpu").manual_seed(seed)
    X = torch.complex(torch.randn(npw, m, generator=g, dtype=torch.float64),
                      torch.randn(npw, m, generator=g, dtype=torch.float64)).to(dev)
    X = X * prec[:, None]

    def H(Y):
        Yt = Y.T.contiguous()
        out = torch.empty_like(Yt)
        gw_apply_h(cell.ctx, Yt, out, GW_FP64)
        return out.T

    def orth(Y):
        Q, R = torch.linalg.qr(Y)
        d = torch.abs(torch.diagonal(R))
        keep = d > 1e-10 * d.max()
        return Q[:, keep]

    X = orth(X)
    P = None
    theta = None
    res = None
    for it in range(max_iter):
        HX = H(X)
        A = X.conj().T @ HX
        A = 0.5 * (A + A.conj().T)
        th, U = torch.linalg.eigh(A)
        X = X @ U
        HX = HX @ U
        R = HX - X * th[None, :]
        res = torch.linalg.vector_norm(R[:, :n + 1], dim=0)
        theta = th
        if verbose and it % 20 == 0:
            print(it, float(res.max()), th[:n + 1].cpu().numpy())
        if float(res.max()) < tol:
            break
        W = R * prec[:, None]
        blocks = [X, W] if P is None else [X, W, P]
        S = orth(torch.cat(blocks, dim=1))
        HS = H(S)
        B = S.conj().T @ HS
        B = 0.5 * (B + B.conj().T)
        w, C = torch.linalg.eigh(B)
        C = C[:, :m]
        Xn = S @ C
        # search direction: the part of the new block outside the old X
        P = Xn - X @ (X.conj().T @ Xn)
        X = orth(Xn)
    eps = theta[:n + 1].cpu().numpy()
    psi = X[:, :n].T.contiguous().cpu().numpy()
    return eps, psi, float(res.max())
