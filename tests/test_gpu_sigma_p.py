"""Parity of the residue term Sigma^P_e(delta) (Eq. pe) on the GPU against the
FP64 oracle, and against the free-electron closed form.

The poles run at real frequencies (SQMR), the seeds are complex in real space
(the states of a dense diagonalisation carry arbitrary phases) or real (a
standing wave), and plane-wave seeds stop the recursion after one step.
Tolerances: FP64 1e-10, mixed 1e-6 (relative to the largest term).
"""
import numpy as np
import pytest

import workloads as W
from oracle import coulomb, pw, sigma_p as SP
from tests.conftest import rel

pytestmark = pytest.mark.gpu

gw = pytest.importorskip("paper_1408_3036_gb300")


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1408_3036_gb300 import _build
    _build.build()
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


@pytest.fixture(scope="module")
def tiny():
    wl = W.tiny()
    c = wl.cells[0]
    sph = pw.Sphere(c.L, c.N, c.ecut)
    gs = pw.ground_state_dense(sph, c.vloc, c.n_occ)
    return c, sph, gs


def _deltas(gs):
    e = gs.eps[-1]
    return [-0.12, 0.0, gs.eps_all[4] - e + 0.03, gs.eps_all[6] - e + 0.01]


@pytest.mark.parametrize("which", [0, 1, 2, 3])
def test_sigma_p_parity(tiny, which):
    """e = HOMO; candidates: the four occupied and four conduction states;
    delta below (three occupied poles), at zero (the HOMO itself, Theta = 1/2)
    and above the gap (two and three conduction poles)."""
    c, sph, gs = tiny
    delta = _deltas(gs)[which]
    C = np.concatenate([gs.C, gs.C_all[4:8]])
    eps = gs.eps_all[:8]
    occ = np.array([1] * 4 + [0] * 4)
    ref_total, ref = SP.sigma_p(gs, gs.C[3], gs.eps[3], delta, C, eps, occ, k=4)
    assert np.count_nonzero(ref) >= 1
    cell = gw.Cell(c.L, c.N, c.ecut, c.vloc, 0)
    cell.set_occupied(gs.C, gs.eps)
    tot, terms = cell.sigma_p(gs.C[3], gs.eps[3], delta, C, eps, occ, k=4, prec=gw.GW_FP64)
    assert np.array_equal(terms == 0.0, ref == 0.0)
    assert rel(terms, ref) < 1e-10
    assert abs(tot - ref_total) < 1e-10 * np.abs(ref).max()
    tot32, terms32 = cell.sigma_p(gs.C[3], gs.eps[3], delta, C, eps, occ, k=4, prec=gw.GW_MIXED)
    assert rel(terms32, ref) < 1e-6
    cell.close()


def test_sigma_p_free_electron_closed_form():
    """V_loc = 0, e = G = 0: conduction plane waves and a standing wave (a real
    seed) give Theta(-w) v(G)/Omega (1/eps~(G, w) - 1), eps~ = 1 - v chi0,
    chi0 = -(2/Omega) |G|^2 / ((|G|^2/2)^2 - w^2); checked without the oracle's
    Sigma^P code.  The seeds are eigenvectors of eps~: one Lanczos step."""
    L, N, ecut = 8.0, 12, 3.0
    sph = pw.Sphere(L, N, ecut)
    cell = gw.Cell(L, N, ecut, np.zeros(sph.ng), 0)

    def unit(n):
        v = np.zeros(sph.npw, complex)
        v[np.nonzero((sph.miller == np.array(n)).all(axis=1))[0][0]] = 1.0
        return v

    cell.set_occupied(unit((0, 0, 0))[None, :], [0.0])
    g2h = 0.5 * (2 * np.pi / L) ** 2
    ns = [(1, 0, 0), (0, 1, 1), (1, 1, 1)]
    C = [unit(n) for n in ns]
    C.append((unit((1, 0, 0)) + unit((-1, 0, 0))) / np.sqrt(2.0))     # cos(G r): real in real space
    C = np.array(C)
    eps = np.array([g2h * 1, g2h * 2, g2h * 3, g2h * 1])
    delta = 2.5 * g2h
    tot, terms = cell.sigma_p(unit((0, 0, 0)), 0.0, delta, C, eps, np.zeros(4, int), k=4, prec=gw.GW_FP64)
    vG = coulomb.vcoul(sph)
    Gn = sph.gvec_norm()
    expect = []
    for n, e in zip(ns + [(1, 0, 0)], eps):
        om = e - delta
        lin = ((n[0] % N) * N + (n[1] % N)) * N + (n[2] % N)
        G2, v = Gn[lin] ** 2, vG[lin]
        chi = -(2.0 / sph.omega_vol) * G2 / ((G2 / 2) ** 2 - om ** 2)
        expect.append(SP.theta(-om) * v / sph.omega_vol * (1.0 / (1.0 - v * chi) - 1.0))
    expect = np.array(expect)
    assert terms[2] == 0.0 and expect[2] == 0.0
    assert rel(terms, expect) < 1e-12
    assert abs(terms[3] - terms[0]) < 1e-12 * abs(terms[0])
    cell.close()


def test_sigma_p_arguments(tiny):
    c, sph, gs = tiny
    cell = gw.Cell(c.L, c.N, c.ecut, c.vloc, 0)
    cell.set_occupied(gs.C, gs.eps)
    C = gs.C_all[4:6]
    with pytest.raises(gw.GwError) as e:
        cell.sigma_p(gs.C[3], gs.eps[3], float("nan"), C, gs.eps_all[4:6], [0, 0])
    assert e.value.status == 7
    with pytest.raises(gw.GwError) as e:
        cell.sigma_p(gs.C[3], gs.eps[3], 0.0, C, gs.eps_all[4:6], [0, 0], k=0)
    assert e.value.status == 1
    tot, terms = cell.sigma_p(gs.C[3], gs.eps[3], -1.0, C, gs.eps_all[4:6], [0, 0])   # no pole
    assert tot == 0.0 and not terms.any()
    cell.close()
