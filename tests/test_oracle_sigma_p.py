"""Pins for the oracle's residue term Sigma^P_e(delta) (Eq. pe).

With V_loc = 0 and plane-wave occupied states, eps~ is diagonal in G and a
seed v^1/2 |p* e> built from plane waves is one of its eigenvectors, so each
term has a closed form and the Lanczos recursion stops after one step.  On a
small cell with a potential, a long recursion reproduces the matrix element
of a dense inverse.
"""
import numpy as np
import pytest

import workloads as W
from oracle import coulomb, pw, response, sigma_p as SP
from tests.conftest import rel


def _free(n_occ, L=8.0, N=12, ecut=3.0):
    sph = pw.Sphere(L, N, ecut)
    gs = pw.ground_state_dense(sph, np.zeros(sph.ng), n_occ)
    return sph, gs


def _pw(sph, n):
    c = np.zeros(sph.npw, complex)
    c[np.nonzero((sph.miller == np.array(n)).all(axis=1))[0][0]] = 1.0
    return c


def test_theta_convention():
    assert SP.theta(0.3) == 1.0 and SP.theta(0.0) == 0.5 and SP.theta(-0.2) == 0.0


def _conduction_closed_form(sph, n, om, wgt):
    vG = coulomb.vcoul(sph)
    Gn = sph.gvec_norm()
    N = sph.N
    lin = ((n[0] % N) * N + (n[1] % N)) * N + (n[2] % N)
    G2, v = Gn[lin] ** 2, vG[lin]
    chi = -(2.0 / sph.omega_vol) * G2 / ((G2 / 2) ** 2 - om ** 2)
    return wgt * v / sph.omega_vol * (1.0 / (1.0 - v * chi) - 1.0)


def test_free_electron_conduction_poles():
    """One occupied state (G = 0, e_e = 0), conduction plane waves c = e^{iGr}.
    For omega_ce = |G|^2/2 - delta <= 0 the term is
        Theta(-omega) v(G)/Omega (1/eps~(G, omega) - 1),
        eps~ = 1 - v(G) chi0(G, omega),  chi0 = -(2/Omega) |G|^2 / ((|G|^2/2)^2 - omega^2),
    and 0 otherwise.  delta = 2.5 (2 pi/L)^2 / 2 puts (1,0,0) and (0,1,1) below
    (no frequency on a transition of the free gas), (1,1,1) and (2,0,0) above;
    a second call with delta on (1,1,1) checks Theta(0) = 1/2."""
    sph, gs = _free(1)
    g2h = 0.5 * (2 * np.pi / sph.L) ** 2
    ns = [(1, 0, 0), (0, 1, 1), (1, 1, 1), (2, 0, 0)]
    C = np.array([_pw(sph, n) for n in ns])
    eps = np.array([g2h * sum(x * x for x in n) for n in ns])
    ce = _pw(sph, (0, 0, 0))
    delta = 2.5 * g2h
    total, terms = SP.sigma_p(gs, ce, 0.0, delta, C, eps, np.zeros(len(ns), int), k=4)
    expect = np.array([_conduction_closed_form(sph, n, e - delta, SP.theta(delta - e)) for n, e in zip(ns, eps)])
    assert terms[2] == 0.0 and terms[3] == 0.0 and expect[0] != 0.0 and expect[1] != 0.0
    assert rel(terms, expect) < 1e-12
    assert abs(total - expect.sum()) < 1e-12 * abs(expect).max()
    # Theta(0) = 1/2: delta on (1,1,1) exactly
    delta = eps[2]
    total, terms = SP.sigma_p(gs, ce, 0.0, delta, C[2:3], eps[2:3], np.zeros(1, int), k=4)
    want = _conduction_closed_form(sph, ns[2], 0.0, 0.5)
    assert want != 0.0 and abs(terms[0] - want) < 1e-12 * abs(want)


def test_free_electron_occupied_poles_closed_shell():
    """Seven occupied plane waves (G = 0 and its six neighbours), e = G = 0,
    delta = -0.05: every occupied state has omega_ve = e_v + 0.05 > 0 and enters
    with weight -1.  The seed v^1/2 |v* e> is the plane wave -G_v, and eps~ is
    diagonal in K with the closed-shell chi0
        chi0(K) = -(2/Omega) sum_v' [K - G_v' in sphere, not occupied] 2D/(D^2 - w^2),
        D = |K - G_v'|^2/2 - |G_v'|^2/2;
    the term of G = 0 itself vanishes (chi0(0) = 0)."""
    sph, gs = _free(7)
    occ = [(0, 0, 0), (1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, 1), (0, 0, -1)]
    C = np.array([_pw(sph, n) for n in occ])
    g2h = 0.5 * (2 * np.pi / sph.L) ** 2
    eps = np.array([g2h * sum(x * x for x in n) for n in occ])
    delta = -0.05
    total, terms = SP.sigma_p(gs, C[0], 0.0, delta, C, eps, np.ones(7, int), k=4)
    sphere_set = {tuple(int(x) for x in m) for m in sph.miller}
    vG = coulomb.vcoul(sph)
    N = sph.N
    expect = np.zeros(7)
    for j, gv in enumerate(occ):
        w_ = eps[j] - delta
        K = tuple(-x for x in gv)
        chi = 0.0
        for gp in occ:
            d = tuple(K[i] - gp[i] for i in range(3))
            if d in sphere_set and d not in occ:
                D = g2h * (sum(x * x for x in d) - sum(x * x for x in gp))
                chi += 2 * D / (D * D - w_ * w_)
        chi *= -(2.0 / sph.omega_vol)
        lin = ((K[0] % N) * N + (K[1] % N)) * N + (K[2] % N)
        v = vG[lin]
        expect[j] = -(v / sph.omega_vol) * (1.0 / (1.0 - v * chi) - 1.0)
    assert expect[0] == 0.0 and abs(terms[0]) < 1e-14
    assert rel(terms, expect) < 1e-12
    assert abs(total - expect.sum()) < 1e-12 * abs(expect).max()


@pytest.mark.parametrize("omega", [0.0, 0.05])
def test_long_recursion_matches_dense_inverse(omega):
    """A cell with a potential: with enough Lanczos steps the pole element
    equals w phi^H (eps~^-1 phi - phi) from a dense solve (complex seed)."""
    wl = W.small(N=8, L=6.0, ecut=2.0, n_occ=2, seed_idx=11)
    c = wl.cells[0]
    sph = pw.Sphere(c.L, c.N, c.ecut)
    gs = pw.ground_state_dense(sph, c.vloc, c.n_occ)
    sqv = np.sqrt(coulomb.vcoul(sph))
    cp = (gs.C_all[3] + 1j * gs.C_all[4]) / np.sqrt(2.0)    # a state complex in real space
    phi = SP.pole_seed(sph, sqv, cp, gs.C[1])
    ph = phi * np.exp(-1j * np.angle(phi[np.argmax(np.abs(phi))]))
    assert np.abs(ph.imag).max() > 1e-2 * np.abs(ph).max()       # not a real field times a phase
    got = SP.pole_element(gs, phi, omega, 120)
    D = response.Dielectric(gs, omega)
    E = D.dense()
    w = sph.omega_vol / sph.ng
    want = (w * np.vdot(phi, np.linalg.solve(E, phi) - phi)).real
    assert abs(got - want) < 1e-10 * abs(want)
    # four steps already give the element to a few parts in 1e4 here
    four = SP.pole_element(gs, phi, omega, 4)
    assert abs(four - want) < 1e-2 * abs(want)
