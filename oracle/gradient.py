"""Derivative of s = <phi|eps~^-1(0)|phi> with respect to V_loc(r_i).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

Not in the paper.  Derivation (pinned by central finite differences in
``tests/test_oracle_gradient.py``):

* ds = -<u|d eps~|u> = <w|d chi0|w>,  u = eps~^-1 phi,  w = v^1/2 u
  (Eq. epsilon: d eps~ = -v^1/2 d chi0 v^1/2).
* chi0 is the second derivative of the band energy E = 2 sum_v e_v with
  respect to the potential, so <w|d chi0|w> along a perturbation z is the
  third derivative E'''[w, w, z].
* Third-order perturbation theory for occupied orbitals (parallel-transport
  gauge, first-order orbitals in P_c):
      T(x, y, z) = sum_v <psi_v^x|V_y|psi_v^z>
                   - sum_{v v'} <psi_v^x|psi_v'^z> <psi_v'|V_y|psi_v>,
      psi_v^x = -G_v P_c V_x psi_v,  G_v = P_c (H - e_v)^-1 P_c,
  E'''[w, w, z] = 2 (2 T(w, z, w) + 4 Re T(w, w, z)) (spin 2, six
  permutations of the symmetric trilinear form).
* With z the Kronecker field at grid point i, <a|z|b> = (Omega/N_g) a*(r_i) b(r_i):
      g1(r) = sum_v |dpsi_v(r)|^2 - sum_{v v'} S_{v v'} psi_v'*(r) psi_v(r)
      eta_v = P_c [w dpsi_v - sum_v' W_{v' v} dpsi_v'],  lambda_v = G_v eta_v
      g2(r) = -sum_v lambda_v*(r) psi_v(r)
      ds/dV_i = (Omega/N_g) (4 g1(r_i) + 8 Re g2(r_i)),
  with dpsi_v = -G_v P_c (w psi_v), S = <dpsi_v|dpsi_v'>, W = <psi_v|w|psi_v'>.
  The resolvents G_v are applied with the dense eigendecomposition.
"""
from __future__ import annotations

import numpy as np

from . import coulomb
from .pw import ground_state_dense, Sphere
from .response import Dielectric, solve_cg


def solve_eps(D: Dielectric, phi, tol=1e-13):
    """u = eps~(0)^-1 phi by CG (eps~(0) is symmetric positive definite, its
    eigenvalues are >= 1: Eq. epsilon_nonp)."""
    u, it, res = solve_cg(lambda x: D.apply(x).real, np.asarray(phi, float), tol)
    return u, it, res


def s_exact(gs, phi, kind=coulomb.TRUNCATED):
    D = Dielectric(gs, 0.0, kind, "sos")
    u, _, _ = solve_eps(D, phi)
    wgt = gs.sph.omega_vol / gs.sph.ng
    return wgt * float(np.dot(phi, u)), u


def grad_vloc(gs, phi, kind=coulomb.TRUNCATED, u=None):
    """ds/dV_i on the grid (dense resolvents)."""
    sph = gs.sph
    vol, ng = sph.omega_vol, sph.ng
    wgt = vol / ng
    D = Dielectric(gs, 0.0, kind, "sos")
    if u is None:
        u, _, _ = solve_eps(D, phi)
    s = wgt * float(np.dot(phi, u))
    w = D.sqrtv(u).real
    U = gs.u                                   # u_v = Omega^1/2 psi_v
    Cc = gs.C_all[gs.n_occ:]
    ec = gs.eps_all[gs.n_occ:]
    nv = gs.n_occ

    def resolvent(v, b):
        """G_v b = sum_c c <c|b> / (e_c - e_v)  (b already in P_c)."""
        a = np.conj(Cc) @ b
        return (a / (ec - gs.eps[v])) @ Cc

    dC = np.array([-resolvent(v, sph.to_sphere(w * U[v])) for v in range(nv)])
    dU = sph.to_grid(dC)                       # Omega^1/2 dpsi_v(r)
    S = np.conj(dC) @ dC.T                     # S[v, v'] = <dpsi_v|dpsi_v'>
    W = (np.conj(U) * w[None, :]) @ U.T / ng   # W[v, v'] = <psi_v|w|psi_v'>
    g1 = (np.sum(np.abs(dU) ** 2, axis=0)
          - np.einsum("ab,br,ar->r", S, np.conj(U), U)).real / vol
    g2 = np.zeros(ng, dtype=np.complex128)
    for v in range(nv):
        eta = sph.to_sphere(w * dU[v]) - W[:, v] @ dC
        eta = eta - (np.conj(gs.C) @ eta) @ gs.C          # P_c
        lam = resolvent(v, eta)
        g2 -= np.conj(sph.to_grid(lam)) * U[v] / vol
    grad = wgt * (4.0 * g1 + 8.0 * g2.real)
    return s, grad, dict(u=u, w=w, dC=dC, g1=g1, g2=g2)


def s_of_v(L, N, ecut, vloc, n_occ, phi, kind=coulomb.TRUNCATED):
    """s for a potential (fresh ground state); used by finite differences."""
    sph = Sphere(L, N, ecut)
    gs = ground_state_dense(sph, vloc, n_occ)
    return s_exact(gs, phi, kind)[0]


def fd_grad(L, N, ecut, vloc, n_occ, phi, points=None, directions=None, h=1e-4,
            kind=coulomb.TRUNCATED):
    """Central finite differences of s at grid points and along directions."""
    vloc = np.asarray(vloc, float)
    out_p, out_d = [], []
    for i in (points if points is not None else []):
        e = np.zeros_like(vloc)
        e[i] = h
        out_p.append((s_of_v(L, N, ecut, vloc + e, n_occ, phi, kind)
                      - s_of_v(L, N, ecut, vloc - e, n_occ, phi, kind)) / (2 * h))
    for d in (directions if directions is not None else []):
        out_d.append((s_of_v(L, N, ecut, vloc + h * d, n_occ, phi, kind)
                      - s_of_v(L, N, ecut, vloc - h * d, n_occ, phi, kind)) / (2 * h))
    return np.array(out_p), np.array(out_d)
