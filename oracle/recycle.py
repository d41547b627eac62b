"""The dielectric matrix at imaginary frequencies from one recycled basis per
occupied state (Sec. "Calculating the dielectric matrix and the integrand at
different frequencies", Eq. recy_eq).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

For fields l (the basis in which eps is expressed), Eq. recy_eq reads
    <l| eps~(i w) - 1 |l'> = 4 sum_v <b_{l,v}| A_v^-1(i w) |b_{l',v}>,
    b_{l,v} = P_c <G| psi_v* v^1/2 l>   (sphere components),
    A_v(i w) = ((H - e_v)^2 + w^2) (H - e_v)^-1.
Per occupied state v the static Sternheimer solutions x_{l,v}(0) =
(H - e_v)^-1 b_{l,v} and the high-frequency directions x_{l,v}(i inf) ~
(H - e_v) b_{l,v} are made into an orthonormal basis gamma_v by a singular
value decomposition; with H_v = gamma^H (H - e_v) gamma and b_gamma =
gamma^H b the operator A_v^-1 is applied in that basis,
    <b|A_v^-1|b'> ~ b_gamma^H H_v (H_v^2 + w^2)^-1 b'_gamma,
so that any number of imaginary frequencies costs only small dense algebra.
Readings: each of the 2 n_l vectors is normalised before the decomposition,
and singular values below rtol times the largest are dropped (rtol = 1e-6 by
default); x(0) is the projected CG solution of the oracle's Sternheimer route.

The same section controls the accuracy of this basis by adding the solutions
x_{l,v}(i w0) at one more frequency (the paper takes w0 = 1 Ha):
    x(i w0) = A_v^-1(i w0) b = ((H - e_v)^2 + w0^2)^-1 (H - e_v) b   (Eq. P2+),
solved here by plain CG on the squared operator, P_c at every step; with
w0 > 0 the basis is built from 3 n_l vectors per state.
"""
from __future__ import annotations

import numpy as np

from . import coulomb
from .pw import h_apply
from .response import project_c, solve_cg, sternheimer_solve


def b_vectors(gs, fields, v, kind=coulomb.TRUNCATED):
    """b_{l,v} = P_c <G| psi_v* v^1/2 l> for every field l (rows)."""
    sph = gs.sph
    sqv = np.sqrt(coulomb.vcoul(sph, kind))
    u = gs.u[v]
    return np.array([project_c(gs, sph.to_sphere(np.conj(u) * coulomb.sqrt_v_apply(sph, sqv, f)))
                     for f in fields])


def x_imag(gs, v, b, w0, tol=1e-14):
    """x(i w0) = ((H - e_v)^2 + w0^2)^-1 (H - e_v) b in the conduction space."""
    sph, vloc, e = gs.sph, gs.vloc, gs.eps[v]

    def Hs(p):
        return project_c(gs, h_apply(sph, vloc, p) - e * p)

    y, _, _ = solve_cg(lambda p: Hs(Hs(p)) + (w0 * w0) * p, Hs(b), tol)
    return project_c(gs, y)


def recycled_basis(gs, v, B, rtol=1e-6, w0=0.0):
    """gamma_v (npw x n_gamma, orthonormal columns) from x(0) and x(i inf),
    and x(i w0) when w0 > 0."""
    sph, vloc, e = gs.sph, gs.vloc, gs.eps[v]
    X0 = [sternheimer_solve(gs, v, 0.0, b, tol=1e-14, gap=1.0) for b in B]
    Xi = [project_c(gs, h_apply(sph, vloc, b) - e * b) for b in B]
    Xw = [x_imag(gs, v, b, w0) for b in B] if w0 > 0 else []
    X = np.array(X0 + Xi + Xw)
    X = X / np.linalg.norm(X, axis=1)[:, None]
    U, s, _ = np.linalg.svd(X.T, full_matrices=False)
    return U[:, s > rtol * s[0]]


def recycle_eps(gs, fields, omegas, kind=coulomb.TRUNCATED, rtol=1e-6, w0=0.0):
    """<l| eps~(i w) - 1 |l'> for every imaginary frequency i w (w in omegas,
    real numbers): array (n_omega, n_l, n_l).  w0 > 0 adds x(i w0) to each
    state's basis."""
    sph, vloc = gs.sph, gs.vloc
    fields = np.atleast_2d(fields)
    out = np.zeros((len(omegas), len(fields), len(fields)))
    for v in range(gs.n_occ):
        B = b_vectors(gs, fields, v, kind)
        gam = recycled_basis(gs, v, B, rtol, w0)
        HG = np.array([h_apply(sph, vloc, g) - gs.eps[v] * g for g in gam.T]).T
        Hv = np.conj(gam.T) @ HG
        bg = np.conj(gam.T) @ B.T
        I = np.eye(len(Hv))
        for o, w in enumerate(omegas):
            K = Hv @ np.linalg.inv(Hv @ Hv + (w * w) * I)
            out[o] += 4.0 * (np.conj(bg.T) @ K @ bg).real
    return out
