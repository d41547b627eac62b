"""The correlation self-energy Sigma^c_e(delta) of Eq. e_c: the frequency
integral of sigma^N - sigma^N0 (Eqs. dge, dg0e), the analytic term Sigma^A
with the Lorentzian model f(w) = alpha^2/(w^2 + alpha^2) (Eqs. he, khe) and
the residue term Sigma^P (Eq. pe).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

Two routes:

* ``sigma_c_plain``: the definitions with the sum over all states n of a dense
  diagonalisation and a dense eps~^-1 (tiny cells):
      sigma^N(i w)  = sum_n <e n*| v^1/2 (eps^-1(i w) - 1) v^1/2 |n* e> w_ne / (w^2 + w_ne^2),
      sigma^N0(i w) = f(w) sum_n <e n*| v^1/2 (eps^-1(0) - 1) v^1/2 |n* e> w_ne / (w^2 + w_ne^2),
      Sigma^A       = sum_n <e n*| v^1/2 (eps^-1(0) - 1) v^1/2 |n* e> F_ne,
  with w_ne = e_n - e_e - delta.
* ``sigma_c_basis``: the paper's evaluation in a basis {l} of fields (Eqs.
  ge, g0e, he, khe): with z_l = Phi_e v^1/2 |l*> (sphere components of
  psi_e(r) (v^1/2 l)(r)), c = e_e + delta and g(h) = h / (w^2 + h^2),
      sigma^N(i w) = sum_ll' M_ll'(i w) <z_l| g(H - c) |z_l'>,  M = eps~^-1 - 1 in {l},
  <z|g(H - c)|z'> from k_h steps of block Lanczos on H - c started with the
  z block (shift-Lanczos: one recursion serves every frequency), M from the
  recycled dielectric matrix (Eq. recy_eq) as (1 + E)^-1 - 1, and
      Sigma^A = 1/2 sum_ll' M_ll'(0) (<z_l| Q_e |h+_l'> + <z_l| P_e |h-_l'>),
      (H - c + alpha) h+ = alpha Q_e z,  (H - c - alpha) h- = alpha P_e z.
The frequency integral uses w = (1 + t)/(1 - t) and Gauss-Legendre nodes in t.

Readings: F_ne = (1/2) alpha / (w_ne + alpha sgn(w_ne)), 0 at w_ne = 0 (the
form Eq. khe gives; the pi in front of Eq. he's F_ne is taken as a typo);
Q_e and P_e hold the states strictly above and below e_e + delta; the basis
route is written for e_HOMO <= c < e_LUMO, where Q_e is the conduction
projector P_c and P_e the occupied states below c.
"""
from __future__ import annotations

import numpy as np

from . import coulomb
from .lanczos import block_lanczos, block_tridiag, _chol_upper
from .pw import h_apply
from .recycle import recycle_eps
from .response import Dielectric, project_c, solve_cg
from .sigma_p import sigma_p


def frequency_nodes(n):
    """Nodes w_i and weights of (1/pi) int_0^inf dw: w = (1 + t)/(1 - t),
    dw = 2 dt / (1 - t)^2, t at the n-point Gauss-Legendre nodes."""
    t, wt = np.polynomial.legendre.leggauss(n)
    return (1.0 + t) / (1.0 - t), wt * 2.0 / (1.0 - t) ** 2 / np.pi


def lorentzian(w, alpha):
    return alpha * alpha / (w * w + alpha * alpha)


def F_ne(w_ne, alpha):
    if w_ne == 0.0:
        return 0.0
    return 0.5 * alpha / (w_ne + alpha * np.sign(w_ne))


def _plain_parts(gs, e, delta, kind):
    """Seeds v^1/2 |n* e> of every state, w_ne, and the elements
    <e n*| v^1/2 (eps^-1(omega) - 1) v^1/2 |n* e> (dense inverse) as a function."""
    sph = gs.sph
    wg = sph.omega_vol / sph.ng
    sqv = np.sqrt(coulomb.vcoul(sph, kind))
    c = gs.eps_all[e] + delta
    u_all = sph.to_grid(gs.C_all)
    ue = u_all[e]
    phis = [coulomb.sqrt_v_apply(sph, sqv, np.conj(u) * ue / sph.omega_vol) for u in u_all]
    wne = gs.eps_all - c

    def elements(omega):
        E = Dielectric(gs, omega, kind).dense()
        Ei = np.linalg.inv(E)
        return np.array([(wg * np.vdot(p, Ei @ p - p)).real for p in phis])

    return phis, wne, elements


def sigma_n_plain(gs, e, delta, w, kind=coulomb.TRUNCATED):
    """sigma^N_e(i w, delta) of Eq. dge by the sum over all states."""
    _, wne, elements = _plain_parts(gs, e, delta, kind)
    return float(np.dot(elements(1j * w if w else 0.0), wne / (w * w + wne * wne)))


def sigma_c_plain(gs, e, delta, alpha, n_freq, kind=coulomb.TRUNCATED):
    """Sigma^c_e(delta) and its parts (integral, Sigma^A, Sigma^P) from the sum
    over all states and dense inverses."""
    sph = gs.sph
    wg = sph.omega_vol / sph.ng
    phis, wne, elements = _plain_parts(gs, e, delta, kind)

    el0 = elements(0.0)
    ws, W = frequency_nodes(n_freq)
    integral = 0.0
    for w, Wt in zip(ws, W):
        elw = elements(1j * w)
        g = wne / (w * w + wne * wne)
        integral += Wt * (np.dot(elw, g) - lorentzian(w, alpha) * np.dot(el0, g))
    SA = sum(el0[n] * F_ne(wne[n], alpha) for n in range(len(wne)))
    SP = 0.0
    for n in range(len(wne)):
        occ = n < gs.n_occ
        th = (1.0 if wne[n] > 0 else 0.5 if wne[n] == 0 else 0.0) if occ else \
             (1.0 if wne[n] < 0 else 0.5 if wne[n] == 0 else 0.0)
        if th == 0.0:
            continue
        if wne[n] == 0.0:
            el = el0[n]
        else:
            Ei = np.linalg.inv(Dielectric(gs, wne[n], kind).dense())
            el = (wg * np.vdot(phis[n], Ei @ phis[n] - phis[n])).real
        SP += (-th if occ else th) * el
    return integral + SA + SP, dict(integral=integral, SA=SA, SP=SP)


def z_vectors(gs, e, fields, kind=coulomb.TRUNCATED):
    """z_l = Phi_e v^1/2 |l*>: sphere components of psi_e(r) (v^1/2 l)(r)."""
    sph = gs.sph
    sqv = np.sqrt(coulomb.vcoul(sph, kind))
    ue = gs.u[e]
    return np.array([sph.to_sphere(ue * coulomb.sqrt_v_apply(sph, sqv, f)) for f in fields])


def g_matrix_lanczos(gs, Z, c, ws, k_h):
    """<z_l| g(H - c, w) |z_l'> for every w from k_h block Lanczos steps on
    H - c started with the rows of Z."""
    sph, vloc = gs.sph, gs.vloc
    As, Bs, _ = block_lanczos(lambda X: np.array([h_apply(sph, vloc, x) - c * x for x in X]), Z, k_h)
    R0 = _chol_upper(np.conj(Z) @ Z.T, False)
    T = block_tridiag(As, Bs)
    th, U = np.linalg.eigh(T)
    b = Z.shape[0]
    U1 = U[:b]
    out = []
    for w in ws:
        G1 = (U1 * (th / (w * w + th * th))) @ np.conj(U1.T)
        out.append(np.conj(R0.T) @ G1 @ R0)
    return out


def g_matrix_dense(gs, Z, c, ws):
    """The same with the dense Hamiltonian (tiny cells)."""
    from .pw import dense_h
    th, V = np.linalg.eigh(dense_h(gs.sph, gs.vloc) - c * np.eye(gs.sph.npw))
    P = np.conj(V.T) @ Z.T
    return [np.conj(P.T) @ ((th / (w * w + th * th))[:, None] * P) for w in ws]


def sigma_c_basis(gs, e, delta, alpha, n_freq, fields, k_h=None, k_p=4, kind=coulomb.TRUNCATED, rtol=1e-6):
    """Sigma^c_e(delta) and its parts in the basis of the (orthonormal, real)
    fields; k_h None uses the dense Hamiltonian for <z|g(H - c)|z'>."""
    sph, vloc = gs.sph, gs.vloc
    c = gs.eps[e] + delta
    if c < gs.eps[-1]:
        raise ValueError("the basis route needs e_HOMO <= e_e + delta")
    fields = np.atleast_2d(fields)
    nl = len(fields)
    ws, W = frequency_nodes(n_freq)
    E = recycle_eps(gs, fields, np.concatenate([[0.0], ws]), kind, rtol)
    I = np.eye(nl)
    M = [np.linalg.inv(I + Ek) - I for Ek in E]
    Z = z_vectors(gs, e, fields, kind)
    G = g_matrix_dense(gs, Z, c, ws) if k_h is None else g_matrix_lanczos(gs, Z, c, ws, k_h)
    integral = 0.0
    for i, Wt in enumerate(W):
        integral += Wt * (np.sum(M[i + 1] * G[i].real) - lorentzian(ws[i], alpha) * np.sum(M[0] * G[i].real))
    # Sigma^A: h+ in the conduction space, h- on the occupied states below c
    Hp = np.zeros((nl, nl))
    for lp in range(nl):
        b = alpha * project_c(gs, Z[lp])
        h, _, _ = solve_cg(lambda x: project_c(gs, h_apply(sph, vloc, x) - (c - alpha) * x), b, 1e-14)
        h = project_c(gs, h)
        for l in range(nl):
            Hp[l, lp] = np.vdot(Z[l], h).real
    a = np.conj(gs.C) @ Z.T                       # <v|z_l>
    Hm = np.zeros((nl, nl))
    for v in range(gs.n_occ):
        if gs.eps[v] < c:
            Hm += (np.outer(np.conj(a[v]), a[v]) * alpha / (gs.eps[v] - c - alpha)).real
    SA = 0.5 * np.sum(M[0] * (Hp + Hm))
    occ = np.ones(gs.n_occ, int)
    SP, _ = sigma_p(gs, gs.C[e], gs.eps[e], delta, gs.C, gs.eps, occ, k=k_p, kind=kind)
    return integral + SA + SP, dict(integral=integral, SA=SA, SP=SP)
