"""Lowest eigenpairs of H = |G|^2/2 + V_loc on the GPU (input preparation).

The method takes the DFT occupied states as input (Sec. Results: ABINIT
ground states converged to squared residual < 1e-12 Ha^2).  For synthetic
cells this module produces them: block LOBPCG whose H applications are the
library's CUDA H-apply (gw_apply_h, FP64).  Tall blocks stay on the device
(torch matmul); the small Gram / Rayleigh-Ritz matrices (a few dozen rows) are
factorised on the host with numpy.  Not part of the dielectric hot path.
"""
from __future__ import annotations

import math

import numpy as np

from . import GW_FP64, gw_apply_h


def _svqb(Y, drop=1e-10):
    """Orthonormal basis of span(Y) (columns), dropping near-dependent
    directions: eigendecomposition of the scaled Gram matrix."""
    import torch
    G = (Y.conj().T @ Y).cpu().numpy()
    d = np.sqrt(np.maximum(np.real(np.diag(G)), 1e-300))
    Gs = G / d[:, None] / d[None, :]
    w, U = np.linalg.eigh(0.5 * (Gs + Gs.conj().T))
    keep = w > drop * w.max()
    T = (U[:, keep] / np.sqrt(w[keep])[None, :]) / d[:, None]
    return Y @ torch.tensor(T, dtype=Y.dtype, device=Y.device)


def _rr(S, HS, m):
    """Rayleigh-Ritz: lowest m Ritz values and coefficient vectors."""
    import torch
    B = (S.conj().T @ HS).cpu().numpy()
    w, C = np.linalg.eigh(0.5 * (B + B.conj().T))
    return w[:m], torch.tensor(C[:, :m], dtype=S.dtype, device=S.device)


def lowest_states(cell, n, tol=1e-10, max_iter=400, extra=None, seed=0, verbose=False, apply=None,
                  device="cuda"):
    """Return (eps[n + 1], psi[n, npw] complex128 numpy, max residual).

    The (n+1)-th eigenvalue is included so that the caller can check the gap
    above the highest occupied state.  ``apply(Yt)`` (rows = vectors) replaces
    the library's H application when given (tests on the host)."""
    import torch
    dev = torch.device(device)
    npw = cell.npw
    m = n + 1 + (extra if extra is not None else max(8, n // 2))
    miller = torch.tensor(cell.sphere(), dtype=torch.float64, device=dev)
    kin = 0.5 * (2 * math.pi / cell.L) ** 2 * (miller ** 2).sum(1)
    prec = 1.0 / (kin + 1.0)
    g = torch.Generator(device="cpu").manual_seed(seed)
    X = torch.complex(torch.randn(npw, m, generator=g, dtype=torch.float64),
                      torch.randn(npw, m, generator=g, dtype=torch.float64)).to(dev)
    X = X * prec[:, None]

    def H(Y):
        Yt = Y.T.contiguous()
        if apply is not None:
            return apply(Yt).T
        out = torch.empty_like(Yt)
        gw_apply_h(cell.ctx, Yt, out, GW_FP64)
        return out.T

    X = _svqb(X)
    P = None
    theta = None
    res = None
    for it in range(max_iter):
        HX = H(X)
        th, U = _rr(X, HX, X.shape[1])
        X = X @ U
        HX = HX @ U
        R = HX - X * torch.tensor(th, device=dev)[None, :]
        res = (R[:, :n + 1].abs() ** 2).sum(0).sqrt()
        theta = th
        if verbose and it % 20 == 0:
            print(it, float(res.max()), th[:n + 1])
        if float(res.max()) < tol:
            break
        # new directions: preconditioned residuals and the previous step,
        # orthogonalised against X (twice) and among themselves
        W = R * prec[:, None]
        Z = W if P is None else torch.cat([W, P], dim=1)
        for _ in range(2):
            Z = Z - X @ (X.conj().T @ Z)
        Qz = _svqb(Z, 1e-14)
        for _ in range(2):
            Qz = Qz - X @ (X.conj().T @ Qz)
        Qz = _svqb(Qz, 1e-14)
        S = torch.cat([X, Qz], dim=1)
        HS = torch.cat([HX, H(Qz)], dim=1)
        w, C = _rr(S, HS, m)
        P = Qz @ C[m:, :]
        X = _svqb(S @ C)
    eps = np.asarray(theta[:n + 1])
    psi = X[:, :n].T.contiguous().cpu().numpy()
    return eps, psi, float(res.max())


def levels_below(cell, emax, n_start, tol=1e-6, max_states=2048, apply=None, device="cuda"):
    """Eigenvalues of H up to ``emax`` (at least ``n_start`` of them), for
    placing frequencies away from the cell's transitions.  Runs the block
    eigensolver with a growing block until its highest converged eigenvalue
    passes ``emax``; the eigenvalues are accurate to about ``tol``.
    ``apply`` and ``device`` as in ``lowest_states``."""
    n = max(int(n_start), 1)
    while True:
        n = min(n, cell.npw - 1, max_states)
        eps, _, _ = lowest_states(cell, n, tol=tol, extra=max(8, n // 4), apply=apply, device=device)
        if eps[-1] > emax or n >= min(cell.npw - 1, max_states):
            return eps[eps <= emax]
        n = 2 * n
