"""Pins for the oracle's correlation self-energy (Eq. e_c).

The basis route (Eqs. ge, g0e, he, khe, recycled eps(i w), shift-Lanczos on
H) equals the definition by the sum over all states with dense inverses when
the basis of fields is complete; block Lanczos on H reproduces g(H - c) once
its Krylov space is the whole sphere; the quadrature and the Lorentzian
analytic term match direct numerical integration.
"""
import numpy as np
import pytest
from scipy import integrate

import workloads as W
from oracle import pw, sigma_c as SC
from tests.conftest import rel


def _cell():
    wl = W.small(N=8, L=6.0, ecut=2.0, n_occ=2, seed_idx=11)
    c = wl.cells[0]
    sph = pw.Sphere(c.L, c.N, c.ecut)
    gs = pw.ground_state_dense(sph, c.vloc, c.n_occ)
    return sph, gs


def test_frequency_nodes_integrate():
    """(1/pi) int_0^inf dw / (1 + w^2) = 1/2 on the mapped Gauss-Legendre nodes."""
    ws, Wt = SC.frequency_nodes(24)
    assert abs(np.sum(Wt / (1.0 + ws * ws)) - 0.5) < 1e-12
    assert (ws > 0).all()


@pytest.mark.parametrize("w_ne", [0.37, -0.21, 2.5])
def test_lorentzian_analytic_term(w_ne):
    """F_ne = (1/pi) int_0^inf f(w) w_ne / (w^2 + w_ne^2) dw with f the
    Lorentzian equals (1/2) alpha / (w_ne + alpha sgn w_ne)."""
    alpha = 1.0
    val, _ = integrate.quad(lambda w: SC.lorentzian(w, alpha) * w_ne / (w * w + w_ne * w_ne), 0, np.inf,
                            epsabs=1e-14, epsrel=1e-13)
    assert abs(val / np.pi - SC.F_ne(w_ne, alpha)) < 1e-12
    assert SC.F_ne(0.0, alpha) == 0.0


def test_block_lanczos_g_matrix_exact_when_complete():
    sph, gs = _cell()
    F = W.random_fields(91, 3, sph.ng)
    Z = SC.z_vectors(gs, 1, F)
    c = gs.eps[1] + 0.01
    ws = [0.05, 0.7, 4.0]
    Gl = SC.g_matrix_lanczos(gs, Z, c, ws, 9)           # 27-dimensional sphere: 9 blocks of 3
    Gd = SC.g_matrix_dense(gs, Z, c, ws)
    for a, b in zip(Gl, Gd):
        assert rel(a, b) < 1e-9


@pytest.mark.parametrize("frac", [0.0, 0.5])
def test_complete_basis_equals_sum_over_states(frac):
    """e = HOMO, delta = frac * gap (delta = 0: the HOMO itself is a pole at
    w = 0 with Theta = 1/2): a complete orthonormal basis of real fields, the
    dense g(H - c) and a long Lanczos for the residue term reproduce the sum
    over all states, part by part."""
    sph, gs = _cell()
    gap = gs.eps_all[gs.n_occ] - gs.eps_all[gs.n_occ - 1]
    delta = frac * gap
    alpha, nf = 1.0, 6
    ref, parts_ref = SC.sigma_c_plain(gs, 1, delta, alpha, nf)
    wg = sph.omega_vol / sph.ng
    F = np.eye(sph.ng) / np.sqrt(wg)
    got, parts = SC.sigma_c_basis(gs, 1, delta, alpha, nf, F, k_h=None, k_p=40)
    for k in ("integral", "SA", "SP"):
        assert abs(parts[k] - parts_ref[k]) < 1e-10 * max(abs(ref), 1e-3), k
    assert abs(got - ref) < 1e-10 * abs(ref)
    if frac == 0.0:
        assert parts_ref["SP"] != 0.0
    else:
        assert parts_ref["SP"] == 0.0


def test_sigma_n_free_electron_closed_form():
    """V_loc = 0, one occupied state (G = 0, e_e = 0): eps~(i w) is diagonal in G
    and <e n*| v^1/2 (eps^-1 - 1) v^1/2 |n* e> = v(G)/Omega (1/eps~(G, i w) - 1)
    for n the plane wave G, with eps~ = 1 - v(G) chi0(G, i w),
    chi0 = -(2/Omega) |G|^2 / ((|G|^2/2)^2 + w^2); so
        sigma^N(i w) = sum_{G != 0} v(G)/Omega (1/eps~ - 1) w_G / (w^2 + w_G^2),
    w_G = |G|^2/2 - delta (the G = 0 term vanishes: chi0(0) = 0)."""
    from oracle import coulomb
    L, N, ecut = 6.0, 8, 2.0
    sph = pw.Sphere(L, N, ecut)
    gs = pw.ground_state_dense(sph, np.zeros(sph.ng), 1)
    delta, w = 0.05, 0.4
    got = SC.sigma_n_plain(gs, 0, delta, w)
    vG = coulomb.vcoul(sph)[sph.index]
    G2 = 2.0 * sph.kin
    m = G2 > 0
    chi = -(2.0 / sph.omega_vol) * G2[m] / ((G2[m] / 2) ** 2 + w * w)
    epsr = 1.0 - vG[m] * chi
    wG = G2[m] / 2 - delta
    want = np.sum(vG[m] / sph.omega_vol * (1.0 / epsr - 1.0) * wG / (w * w + wG * wG))
    assert abs(got - want) < 1e-12 * abs(want)


def test_sigma_c_independent_of_the_model_width():
    """The Lorentzian model is subtracted under the integral and added back as
    Sigma^A (Eqs. e_c, dhe): with enough frequency nodes the total does not
    depend on alpha, while the parts do."""
    sph, gs = _cell()
    delta = 0.3 * (gs.eps_all[gs.n_occ] - gs.eps_all[gs.n_occ - 1])
    a, pa = SC.sigma_c_plain(gs, 1, delta, 0.5, 48)
    b, pb = SC.sigma_c_plain(gs, 1, delta, 2.0, 48)
    assert abs(pa["SA"] - pb["SA"]) > 1e-3 * abs(a)
    assert abs(a - b) < 1e-7 * abs(a)
