"""Pins for the oracle's model operator (Sec. Dielectric model, Eq. model_eq)
and for the split of eps^-1 - 1 over an exact and a model basis (Eq.
subs_epsilon).

The model replaces H by the kinetic operator T in Eq. P2a.  Where the
occupied states are plane waves (V_loc constant) the projector on the
conduction space is diagonal in G and every quantity has a closed form; at
V_loc = 0 the model and the exact operator coincide (H = T), and the exact
operator is pinned independently by the sum over states (Eq. P) and its own
closed forms.
"""
import numpy as np
import pytest

import workloads as W
from oracle import coulomb, lanczos, pw, response
from tests.conftest import rel


def _field(n, seed=3, complex_=False):
    return W.random_fields(seed, 1, n, complex_)[0]


def _uniform(V0, n_occ, L=8.0, N=12, ecut=3.0):
    sph = pw.Sphere(L, N, ecut)
    gs = pw.ground_state_dense(sph, np.full(sph.ng, V0), n_occ)
    return sph, gs


@pytest.mark.parametrize("n_occ", [1, 7])
@pytest.mark.parametrize("omega", [0.0, 0.05, 0.1 + 0.2j])
def test_model_equals_exact_for_free_electrons(n_occ, omega):
    """V_loc = 0: H = T, so Eq. model_eq is chi0 itself (G = 0, or G = 0 and
    its six neighbours, occupied)."""
    sph, gs = _uniform(0.0, n_occ)
    f = _field(sph.ng, 21, complex_=True)
    assert rel(response.chi0_model(gs, f, omega), response.chi0_sos(gs, f, omega)) < 1e-12


@pytest.mark.parametrize("omega", [0.0, 0.05, 0.1 + 0.2j])
def test_model_constant_potential_closed_form(omega):
    """V_loc = V0, one occupied state (G = 0, e_0 = V0): the model is diagonal
    in G with
        P~(G) = -(2/Omega) [1/(|G|^2/2 - V0 - omega) + 1/(|G|^2/2 - V0 + omega)]
    for G != 0 in the sphere, while chi0 does not depend on V0.  Pins the
    absolute e_v in the kinetic denominators, both signs, the spin factor and
    the normalisation."""
    V0 = -0.37
    sph, gs = _uniform(V0, 1)
    assert abs(gs.eps[0] - V0) < 1e-12
    f = _field(sph.ng, 22, complex_=True)
    G2 = sph.gvec_norm() ** 2
    insph = np.zeros(sph.ng, bool)
    insph[sph.index] = True
    m = insph & (G2 > 0)
    expect = np.zeros(sph.ng, complex)
    t = G2[m] / 2 - V0
    expect[m] = -(2.0 / sph.omega_vol) * (1.0 / (t - omega) + 1.0 / (t + omega))
    model = response.chi0_model(gs, f, omega)
    assert rel(sph.fwd(model), expect * sph.fwd(f)) < 1e-12
    # chi0 is invariant under the shift, the model is not
    sph0, gs0 = _uniform(0.0, 1)
    exact = response.chi0_sos(gs, f, omega)
    assert rel(exact, response.chi0_sos(gs0, f, omega)) < 1e-12
    assert rel(model, exact) > 1e-2


def test_model_closed_shell_constant_potential():
    """V_loc = V0, seven occupied states (G = 0 and its six neighbours): the
    conduction projector removes K - G_v whenever that is an occupied wave
    vector, and
        P~(K) = -(2/Omega) sum_v [K - G_v in sphere, not occupied]
                * (1/(D_v - omega) + 1/(D_v + omega)),
        D_v = |K - G_v|^2/2 - (|G_v|^2/2 + V0),
    with K - G_v wrapped into the grid (products of grid fields alias)."""
    V0 = 0.21
    sph, gs = _uniform(V0, 7)
    N = sph.N
    occ = [(0, 0, 0), (1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, 1), (0, 0, -1)]
    g = 2 * np.pi / sph.L
    sphere_set = {tuple(int(x) for x in m) for m in sph.miller}
    n = pw.fft_n(N)
    omega = 0.07
    expect = np.zeros((N, N, N), complex)
    for i0 in range(N):
        for i1 in range(N):
            for i2 in range(N):
                tot = 0.0
                for gv in occ:
                    d = (n[i0] - gv[0], n[i1] - gv[1], n[i2] - gv[2])
                    d = tuple(int(n[x % N]) for x in d)
                    if d in sphere_set and d not in occ:
                        D = 0.5 * g * g * (sum(x * x for x in d) - sum(x * x for x in gv)) - V0
                        tot += 1.0 / (D - omega) + 1.0 / (D + omega)
                expect[i0, i1, i2] = -(2.0 / sph.omega_vol) * tot
    f = _field(sph.ng, 23, complex_=True)
    got = sph.fwd(response.chi0_model(gs, f, omega))
    assert rel(got, expect.reshape(-1) * sph.fwd(f)) < 1e-12


def test_model_symmetry_and_sign(small_case):
    """General V_loc: the model is Hermitian at real omega (and maps real
    fields to real fields, the occupied space being closed under
    conjugation), complex symmetric in the bilinear form at complex omega, and
    negative semidefinite at omega = 0 when every e_v < 0 (then each kinetic
    denominator is positive)."""
    _, c, sph, gs = small_case
    assert (gs.eps < 0).all()
    f, h = W.random_fields(31, 2, sph.ng)
    w = sph.omega_vol / sph.ng
    for omega in (0.0, 0.3):
        Pf = response.chi0_model(gs, f, omega)
        Ph = response.chi0_model(gs, h, omega)
        assert np.abs(Pf.imag).max() < 1e-13 * np.abs(Pf).max()
        assert abs(np.vdot(h, Pf) - np.vdot(Ph, f)) < 1e-13 * abs(np.vdot(h, Pf))
    omega = 0.3 + 0.1j
    Pf = response.chi0_model(gs, f, omega)
    Ph = response.chi0_model(gs, h, omega)
    assert abs(np.sum(h * Pf) - np.sum(Ph * f)) < 1e-13 * abs(np.sum(h * Pf))
    for s in range(4):
        x = W.random_fields(40 + s, 1, sph.ng)[0]
        assert w * np.vdot(x, response.chi0_model(gs, x, 0.0)).real < 0.0


def _split_cell():
    wl = W.small(N=8, L=6.0, ecut=2.0, n_occ=2, seed_idx=11)
    c = wl.cells[0]
    sph = pw.Sphere(c.L, c.N, c.ecut)
    gs = pw.ground_state_dense(sph, c.vloc, c.n_occ)
    assert gs.gap() > 1e-3 and (gs.eps < 0).all()
    return c, sph, gs


def test_split_complete_basis_is_exact():
    """In a complete orthonormal basis of the real fields (both bases), the two
    parts of Eq. subs_epsilon add up to <phi|eps^-1 - 1|phi>, taken here by a
    dense solve with the exact operator (sum over states)."""
    c, sph, gs = _split_cell()
    w = sph.omega_vol / sph.ng
    D = response.Dielectric(gs, 0.0, route="sos")
    Dm = response.Dielectric(gs, 0.0, route="model")
    Q = np.eye(sph.ng) / np.sqrt(w)
    T = lanczos.compress(lambda x: D.apply(x), Q, w).real
    M = lanczos.compress(lambda x: Dm.apply(x), Q, w).real
    phi = W.random_fields(51, 2, sph.ng)
    a = w * phi @ Q.T
    got = lanczos.epsinv_split(a, T, M, a, M)
    E = D.dense().real
    want = w * phi @ (np.linalg.solve(E, phi.T) - phi.T)
    assert rel(got, want) < 1e-11
    # the model part alone is not the answer: the first part matters
    assert rel(a @ (np.linalg.inv(M) - np.eye(len(M))) @ a.T, want) > 1e-3


def test_split_reduces_to_plain_lanczos_when_model_is_exact():
    """V_loc = 0 (the model equals the exact operator): the Lanczos bases of
    the two operators coincide, M = T, the first part vanishes and the split is
    the plain Lanczos estimate |phi|^2 ((T^-1)_11 - 1)."""
    sph, gs = _uniform(0.0, 1, L=6.0, N=8, ecut=2.0)
    w = sph.omega_vol / sph.ng
    D = response.Dielectric(gs, 0.0, route="sos")
    Dm = response.Dielectric(gs, 0.0, route="model")
    phi = W.random_fields(52, 1, sph.ng)[0]
    k = 6
    al, be, Q = lanczos.lanczos(lambda x: D.apply(x), phi, k, weight=w)
    alm, bem, Qm = lanczos.lanczos(lambda x: Dm.apply(x), phi, k, weight=w)
    assert np.abs(np.array(al) - np.array(alm)).max() < 1e-12
    T = lanczos.tridiag(al, be)
    M = lanczos.compress(lambda x: Dm.apply(x), Q, w).real
    assert np.abs(M - T).max() < 1e-12
    a = w * np.array(Q) @ phi
    am = w * np.array(Qm) @ phi
    got = lanczos.epsinv_split(a[None], T, M, am[None], lanczos.tridiag(alm, bem))[0, 0]
    nrm2 = w * phi @ phi
    assert abs(got - nrm2 * (np.linalg.inv(T)[0, 0] - 1.0)) < 1e-12 * nrm2
