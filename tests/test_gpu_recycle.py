"""Parity of the recycled-basis dielectric matrix at imaginary frequencies
(Eq. recy_eq) on the GPU: against the oracle's recycling (same algorithm), and
against the exact matrix from the sum over states where the method is exact
(w = 0; a recycled basis spanning the conduction space)."""
import numpy as np
import pytest

import workloads as W
from oracle import pw, recycle, response
from tests.conftest import rel

pytestmark = pytest.mark.gpu

gw = pytest.importorskip("paper_1408_3036_gb300")

WS = [0.0, 0.1, 0.5, 2.0, 10.0]


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1408_3036_gb300 import _build
    _build.build()
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _setup(wl):
    c = wl.cells[0]
    sph = pw.Sphere(c.L, c.N, c.ecut)
    gs = pw.ground_state_dense(sph, c.vloc, c.n_occ)
    cell = gw.Cell(c.L, c.N, c.ecut, c.vloc, 0)
    cell.set_occupied(gs.C, gs.eps)
    return c, sph, gs, cell


def _exact(gs, F, w):
    D = response.Dielectric(gs, 1j * w if w else 0.0)
    wg = gs.sph.omega_vol / gs.sph.ng
    return np.array([[(wg * np.dot(F[i], D.apply(F[j], real=False) - F[j])).real for j in range(len(F))]
                     for i in range(len(F))])


def test_recycle_parity_small():
    c, sph, gs, cell = _setup(W.small())
    F = W.random_fields(71, 4, sph.ng)
    ref = recycle.recycle_eps(gs, F, WS)
    got, kept = cell.recycle_eps(F, WS, prec=gw.GW_FP64)
    assert kept == 8
    assert rel(got, ref) < 1e-10
    assert rel(got[0], _exact(gs, F, 0.0)) < 1e-10          # exact at w = 0
    got32, _ = cell.recycle_eps(F, WS, prec=gw.GW_MIXED)
    assert rel(got32, ref) < 1e-6
    cell.close()


def test_recycle_parity_tiny_more_fields():
    """Four occupied states, 534 plane waves, six fields (grid 16^3)."""
    c, sph, gs, cell = _setup(W.tiny())
    F = W.random_fields(72, 6, sph.ng)
    ref = recycle.recycle_eps(gs, F, WS)
    got, kept = cell.recycle_eps(F, WS, prec=gw.GW_FP64)
    assert kept == 12
    assert rel(got, ref) < 1e-10
    cell.close()


def test_recycle_complete_basis_exact():
    """27 plane waves, 2 occupied, 16 fields: the recycled vectors span the
    25-dimensional conduction space; exact at every imaginary frequency."""
    c, sph, gs, cell = _setup(W.small(N=8, L=6.0, ecut=2.0, n_occ=2, seed_idx=11))
    assert sph.npw == 27
    F = W.random_fields(62, 16, sph.ng)
    got, kept = cell.recycle_eps(F, WS, prec=gw.GW_FP64)
    assert kept == 25
    for o, w in enumerate(WS):
        assert rel(got[o], _exact(gs, F, w)) < 1e-10
    cell.close()


def test_recycle_arguments():
    c, sph, gs, cell = _setup(W.small())
    F = W.random_fields(73, 2, sph.ng)
    with pytest.raises(gw.GwError) as e:
        cell.recycle_eps(F, [0.1, float("nan")])
    assert e.value.status == 7
    with pytest.raises(gw.GwError) as e:
        cell.recycle_eps(F, [0.1], rtol=2.0)
    assert e.value.status == 1
    cell.set_operator(gw.GW_OP_MODEL)
    with pytest.raises(gw.GwError) as e:
        cell.recycle_eps(F, [0.1])
    assert e.value.status == 8
    cell.close()


def test_recycle_augmented_parity():
    """Bases augmented with x(i w0), w0 = 1 Ha (the recycling section's accuracy
    control): equal to the oracle's augmented recycling (FP64 1e-10, mixed
    1e-6), 3 nl directions kept per state, and closer to the exact matrix than
    the plain basis at w = 0.5 and 2 Ha."""
    c, sph, gs, cell = _setup(W.small())
    F = W.random_fields(71, 4, sph.ng)
    ref = recycle.recycle_eps(gs, F, WS, w0=1.0)
    plain, _ = cell.recycle_eps(F, WS, prec=gw.GW_FP64)
    cell.set_recycle_augment(1.0)
    got, kept = cell.recycle_eps(F, WS, prec=gw.GW_FP64)
    assert kept == 12
    assert rel(got, ref) < 1e-10
    got32, _ = cell.recycle_eps(F, WS, prec=gw.GW_MIXED)
    assert rel(got32, ref) < 1e-6
    assert rel(got[WS.index(2.0)], _exact(gs, F, 2.0)) < rel(plain[WS.index(2.0)], _exact(gs, F, 2.0))
    assert rel(got[WS.index(0.5)], _exact(gs, F, 0.5)) < rel(plain[WS.index(0.5)], _exact(gs, F, 0.5))
    cell.close()
