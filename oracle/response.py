"""Independent-particle response chi0(omega) and the symmetric dielectric
operator eps~ = 1 - v^1/2 chi0 v^1/2.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

Three routes to chi0 f for a grid field f (all give the same result up to
rounding; the tests pin them against each other and against closed forms),
and a fourth, different operator, the model polarizability of Sec. Dielectric
model (Eq. model_eq, ``chi0_model``, route "model" of ``Dielectric``):

1. ``chi0_eqP``: Eq. P literally,
       P(w) = 2 sum_{c,v} |c* v> [1/(w - (e_c - e_v)) - 1/(w + (e_c - e_v))] <v c*|
   with the grid functions psi_c*(r) psi_v(r) and the grid inner product.
   The factor 2 is spin (non-spin-polarised, Sec. The G0W0 method).
2. ``chi0_sos``: Eq. P1 with Eq. fvpm written in the plane-wave basis,
       chi0 f = -2 sum_v psi_v (x_v^- + x_v^+),
       x_v^(-/+) = sum_c psi_c <psi_c|psi_v* f> / (e_c - e_v -/+ w).
   Equal to route 1 because H is real in real space, so the occupied and
   conduction spaces are closed under complex conjugation (c -> c* relabels
   the conduction sum).  This analytic form is also the one used at complex w.
3. ``chi0_sternheimer``: Eq. P2, solving (H - e_v -/+ w) x_v^(-/+) = P_c psi_v* f
   iteratively in the plane-wave sphere, projecting on the conduction space at
   every step (Sec. Avoiding summations, the paragraph after the SQMR footnote).

The symmetric operator is Eq. epsilon: eps~ x = x - v^1/2 chi0 v^1/2 x.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse.linalg

from . import coulomb
from .pw import h_apply


# ---------------------------------------------------------------------------
# Route 1: Eq. P, literal
# ---------------------------------------------------------------------------
def chi0_eqP(gs, f, omega, chunk=256):
    """(P(omega) f)(r) by Eq. P with every conduction state of a dense
    diagonalisation.  f: (N_g,) grid field (real or complex)."""
    sph = gs.sph
    if gs.C_all is None:
        raise ValueError("Eq. P needs all eigenstates (dense ground state)")
    vol = sph.omega_vol
    wgt = vol / sph.ng
    psi_all = sph.to_grid(gs.C_all) / np.sqrt(vol)       # psi_n(r)
    nv = gs.n_occ
    out = np.zeros(sph.ng, dtype=np.complex128)
    for v in range(nv):
        for a in range(nv, len(gs.eps_all), chunk):
            cs = slice(a, min(a + chunk, len(gs.eps_all)))
            pair = np.conj(psi_all[cs]) * psi_all[v][None, :]   # |c* v>
            coeff = wgt * (np.conj(pair) @ f)                    # <v c*|f>
            d = gs.eps_all[cs] - gs.eps_all[v]
            w = 2.0 * (1.0 / (omega - d) - 1.0 / (omega + d))
            out += (w * coeff) @ pair
    return out


# ---------------------------------------------------------------------------
# Route 2: Eqs. P1 + fvpm in the plane-wave basis (dense resolvent)
# ---------------------------------------------------------------------------
def chi0_sos(gs, f, omega):
    sph = gs.sph
    if gs.C_all is None:
        raise ValueError("sum over states needs all eigenstates")
    vol = sph.omega_vol
    u = gs.u
    Cc = gs.C_all[gs.n_occ:]                 # (ncond, npw)
    ec = gs.eps_all[gs.n_occ:]
    out = np.zeros(sph.ng, dtype=np.complex128)
    for v in range(gs.n_occ):
        g = sph.to_sphere(np.conj(u[v]) * f)         # <G|psi_v* f>
        a = np.conj(Cc) @ g                          # <psi_c|psi_v* f>
        d = ec - gs.eps[v]
        xm = (a / (d - omega)) @ Cc                  # x_v^-
        xp = (a / (d + omega)) @ Cc                  # x_v^+
        out += u[v] * sph.to_grid(xm + xp)
    return -2.0 / vol * out


# ---------------------------------------------------------------------------
# Route 3: Sternheimer equations (Eq. P2) solved iteratively
# ---------------------------------------------------------------------------
def project_c(gs, y):
    """P_c y = y - sum_v c_v <c_v|y> in the sphere."""
    return y - (np.conj(gs.C) @ y) @ gs.C


def solve_cg(apply_A, b, tol=1e-14, maxiter=20000, atol=0.0, stall=500):
    """Textbook conjugate gradients for a Hermitian positive definite A, until
    |r| <= max(tol |b|, atol).  In floating point the recursion can reach a
    floor above that target (a right-hand side much smaller than the rounding
    of its own construction); it then stops once |r| has not halved in
    `stall` iterations and returns the iterate of smallest |r| seen.
    Returns (x, iterations, relative residual of that iterate)."""
    x = np.zeros_like(b)
    r = b.copy()
    p = r.copy()
    rr = np.vdot(r, r).real
    bb = rr
    if bb == 0.0:
        return x, 0, 0.0
    stop2 = max(tol * tol * bb, atol * atol)
    best, x_best, it_best = rr, x.copy(), 0
    it = 0
    while rr > stop2 and it < maxiter and it - it_best <= stall:
        Ap = apply_A(p)
        alpha = rr / np.vdot(p, Ap).real
        x = x + alpha * p
        r = r - alpha * Ap
        rr_new = np.vdot(r, r).real
        p = r + (rr_new / rr) * p
        rr = rr_new
        it += 1
        if rr < best:
            if rr < 0.25 * best:
                it_best = it
            best, x_best = rr, x.copy()
    return x_best, it, np.sqrt(best / bb)


def solve_general(apply_A, b, tol=1e-13, atol=0.0):
    """Non-Hermitian-positive cases (indefinite or complex shift): GMRES
    (library routine) on the same projected operator."""
    n = b.shape[0]
    A = scipy.sparse.linalg.LinearOperator((n, n), matvec=apply_A,
                                           dtype=np.complex128)
    x, info = scipy.sparse.linalg.gmres(A, b, rtol=tol, atol=atol,
                                        restart=min(n, 400), maxiter=200)
    if info != 0:
        raise RuntimeError(f"gmres did not converge ({info})")
    return x


def sternheimer_solve(gs, v, shift, b, tol=1e-14, gap=None, atol=0.0):
    """Solve (H - e_v + shift) x = b in the conduction space (Eq. P2 with
    shift = -/+ omega), P_c applied at every iteration, until the residual is
    below max(tol |b|, atol)."""
    sph, vloc = gs.sph, gs.vloc
    e = gs.eps[v]

    def A(p):
        return project_c(gs, h_apply(sph, vloc, p) - (e - shift) * p)

    hpd = (np.imag(shift) == 0.0) and (gap is not None) and (np.real(shift) > -gap)
    if hpd:
        x, _, _ = solve_cg(A, b, tol, atol=atol)
    else:
        x = solve_general(A, b, tol, atol=atol)
    return project_c(gs, x)


def chi0_sternheimer(gs, f, omega, tol=1e-14, gaps=None, states=None):
    """chi0 f by Eq. P2: two Sternheimer solves per occupied state (one when
    omega = 0, where x^- = x^+).  ``states`` restricts the sum over occupied
    states to a subset (a partial sum, for timing samples only)."""
    sph = gs.sph
    vol = sph.omega_vol
    u = gs.u
    out = np.zeros(sph.ng, dtype=np.complex128)
    for v in (range(gs.n_occ) if states is None else states):
        # The target is relative to psi_v* f before P_c: the projected right-hand
        # side carries rounding of that size, so a target relative to b alone
        # is out of reach when P_c removes most of psi_v* f (the paper's own
        # criterion is absolute, Sec. Results).
        g = sph.to_sphere(np.conj(u[v]) * f)
        b = project_c(gs, g)
        atol = tol * np.linalg.norm(g)
        gap = None if gaps is None else gaps[v]
        xm = sternheimer_solve(gs, v, -omega, b, tol, gap, atol)
        if omega == 0:
            xs = 2.0 * xm
        else:
            xs = xm + sternheimer_solve(gs, v, +omega, b, tol, gap, atol)
        out += u[v] * sph.to_grid(xs)
    return -2.0 / vol * out


def conduction_gaps(gs, lowest_conduction):
    """Per occupied state v: e_c(lowest) - e_v (CG applies to (H - e_v - w) on
    P_c while w < this gap)."""
    return lowest_conduction - gs.eps


# ---------------------------------------------------------------------------
# Route 4: the model operator of Sec. Dielectric model (Eq. model_eq)
# ---------------------------------------------------------------------------
def chi0_model(gs, f, omega):
    """P~(omega) f of Eq. model_eq: Eq. P2a with H replaced by the kinetic
    operator T, which is diagonal in the plane-wave sphere.  Per occupied
    state v,
        b        = P_c <G|psi_v* f>
        f~_v(-/+) = P_c [ b / (|G|^2/2 - e_v -/+ omega) ]
    and, as in Eq. P1, P~ f = -2 sum_v psi_v (f~_v(-) + f~_v(+)).
    The energies are the absolute e_v of the occupied states (the model is not
    invariant under a constant shift of V_loc, unlike chi0).
    Reading: where a denominator is exactly zero its reciprocal is taken as 0
    (the pseudo-inverse of the diagonal).  That happens on an occupied plane
    wave of a free-electron cell, where P_c b vanishes; elsewhere the model,
    like chi0, is singular at such a real frequency."""
    sph = gs.sph
    vol = sph.omega_vol
    u = gs.u

    def pinv(d):
        out = np.zeros_like(d, dtype=np.complex128)
        nz = d != 0
        out[nz] = 1.0 / d[nz]
        return out

    out = np.zeros(sph.ng, dtype=np.complex128)
    for v in range(gs.n_occ):
        b = project_c(gs, sph.to_sphere(np.conj(u[v]) * f))
        xm = project_c(gs, b * pinv(sph.kin - gs.eps[v] - omega))
        xp = project_c(gs, b * pinv(sph.kin - gs.eps[v] + omega))
        out += u[v] * sph.to_grid(xm + xp)
    return -2.0 / vol * out


# ---------------------------------------------------------------------------
# Eq. P2+: squared Hermitian form at imaginary frequency
# ---------------------------------------------------------------------------
def f_sum_imag(gs, v, f, w_im, tol=1e-14):
    """Solve ((H - e_v)^2 + w^2) y = 2 (H - e_v) P_c psi_v* f (Eq. P2+ with
    omega = i w); the solution is x^- + x^+ at omega = i w (Eq. fv)."""
    sph, vloc = gs.sph, gs.vloc
    e = gs.eps[v]

    def Hs(p):
        return project_c(gs, h_apply(sph, vloc, p) - e * p)

    b = project_c(gs, sph.to_sphere(np.conj(gs.u[v]) * f))
    rhs = 2.0 * Hs(b)
    y, _, _ = solve_cg(lambda p: Hs(Hs(p)) + (w_im * w_im) * p, rhs, tol)
    return project_c(gs, y)


# ---------------------------------------------------------------------------
# Eq. epsilon: the symmetric dielectric operator
# ---------------------------------------------------------------------------
class Dielectric:
    """eps~(omega) x = x - v^1/2 chi0(omega) v^1/2 x with a chosen chi0 route
    (route "model": the model operator eps~_model of Eq. model_eq)."""

    def __init__(self, gs, omega=0.0, kind=coulomb.TRUNCATED, route="sos",
                 tol=1e-14, gaps=None):
        self.gs, self.omega, self.route, self.tol = gs, omega, route, tol
        self.sqv = np.sqrt(coulomb.vcoul(gs.sph, kind))
        self.gaps = gaps

    def chi0(self, f):
        if self.route == "eqP":
            return chi0_eqP(self.gs, f, self.omega)
        if self.route == "sos":
            return chi0_sos(self.gs, f, self.omega)
        if self.route == "sternheimer":
            return chi0_sternheimer(self.gs, f, self.omega, self.tol, self.gaps)
        if self.route == "model":
            return chi0_model(self.gs, f, self.omega)
        raise ValueError(self.route)

    def sqrtv(self, x):
        return coulomb.sqrt_v_apply(self.gs.sph, self.sqv, x)

    def apply(self, x, real=None):
        y = self.sqrtv(x)
        dn = self.chi0(y)
        out = x - self.sqrtv(dn)
        if real is None:
            real = np.isrealobj(x) and np.imag(self.omega) == 0
        return out.real if real else out

    def dense(self):
        """eps~ as an N_g x N_g matrix, one column per grid point (tiny cells)."""
        ng = self.gs.sph.ng
        E = np.empty((ng, ng), dtype=np.complex128)
        for j in range(ng):
            e = np.zeros(ng)
            e[j] = 1.0
            E[:, j] = self.apply(e, real=False)
        return E
