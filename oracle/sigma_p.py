"""Residue term Sigma^P_e(delta) of the correlation self-energy (Eq. pe) from
one short Lanczos recursion per pole (Sec. "Calculating the dielectric matrix
and the integrand at different frequencies").

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

Eq. pe, with omega_ne = e_n - e_e - delta and <r|n* e> = psi_n(r)* psi_e(r):
    Sigma^P_e(delta) = - sum_v <e v*| v^1/2 (eps^-1(omega_ve) - 1) v^1/2 |v* e> Theta(omega_ve)
                       + sum_c <e c*| v^1/2 (eps^-1(omega_ce) - 1) v^1/2 |c* e> Theta(-omega_ce)
(v occupied, c conduction; Theta(0) = 1/2).  Each matrix element is taken
from a Lanczos recursion on eps~(omega_pe) seeded with phi = v^1/2 |p* e>:
    <phi| eps~^-1 - 1 |phi> ~ |phi|^2 ((T_k^-1)_11 - 1),
k steps (four converge the term to 1 meV in the paper), stopping early at an
invariant subspace.
"""
from __future__ import annotations

import numpy as np

from . import coulomb
from .lanczos import lanczos, tridiag
from .response import Dielectric


def theta(x):
    """Step function with Theta(0) = 1/2."""
    return 1.0 if x > 0 else (0.5 if x == 0 else 0.0)


def pole_seed(sph, sqv, c_p, c_e):
    """phi = v^1/2 |p* e> on the grid from sphere coefficients (psi = Omega^-1/2
    sum_G c_G e^{iGr})."""
    f = np.conj(sph.to_grid(c_p)) * sph.to_grid(c_e) / sph.omega_vol
    return coulomb.sqrt_v_apply(sph, sqv, f)


def pole_element(gs, phi, omega, k, kind=coulomb.TRUNCATED, route="sos", breakdown=1e-14):
    """<phi| eps~^-1(omega) - 1 |phi> from k Lanczos steps seeded with phi."""
    sph = gs.sph
    w = sph.omega_vol / sph.ng
    n2 = w * np.vdot(phi, phi).real
    if n2 == 0.0:
        return 0.0
    D = Dielectric(gs, omega, kind, route)
    al, be, _ = lanczos(lambda x: D.apply(x, real=False), phi, k, weight=w, breakdown=breakdown)
    Ti = np.linalg.inv(tridiag(al, be))
    return float((n2 * (Ti[0, 0] - 1.0)).real)


def sigma_p(gs, c_e, eps_e, delta, C, eps, occ, k=4, kind=coulomb.TRUNCATED, route="sos"):
    """Sigma^P_e(delta) and the signed term of every state (0 where Theta
    excludes it).  C: (n, npw) sphere coefficients of the candidate pole
    states, eps their energies, occ 1 for occupied, 0 for conduction."""
    sph = gs.sph
    sqv = np.sqrt(coulomb.vcoul(sph, kind))
    terms = np.zeros(len(eps))
    for p in range(len(eps)):
        om = eps[p] - eps_e - delta
        wgt = -theta(om) if occ[p] else theta(-om)
        if wgt == 0.0:
            continue
        phi = pole_seed(sph, sqv, C[p], c_e)
        terms[p] = wgt * pole_element(gs, phi, om, k, kind, route)
    return float(terms.sum()), terms
