"""Parity of the GPU adjoint (gw_grad_vloc) with the oracle's gradient of
s = <phi|eps~^-1(0)|phi> (itself pinned by central finite differences)."""
import numpy as np
import pytest

import workloads as W
from oracle import gradient, pw
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


def _case(wl, centre):
    c = wl.cells[0]
    sph = pw.Sphere(c.L, c.N, c.ecut)
    gs = pw.ground_state_dense(sph, c.vloc, c.n_occ)
    phi = W.gaussian_phi(c.L, c.N, centre)
    return c, sph, gs, phi


@pytest.mark.parametrize("prec,tol", [(0, 1e-9), (1, 1e-6)])
def test_gradient_small(prec, tol):
    c, sph, gs, phi = _case(W.small(), [1.0, 2.0, 3.0])
    s_ref, g_ref, _ = gradient.grad_vloc(gs, phi)
    cell = gw.Cell(c.L, c.N, c.ecut, c.vloc)
    cell.set_occupied(gs.C, gs.eps)
    s, g = cell.grad_vloc(phi, 30, prec)
    cell.close()
    assert abs(s - s_ref) < tol * abs(s_ref)
    assert rel(g, g_ref) < tol
    assert abs(g.sum()) < 10 * tol * np.abs(g).sum()


def test_gradient_differentiation_config():
    """Differentiation config (32^3, N_occ = 8, K = 40): FP64 and mixed."""
    wl = W.differentiation()
    c = wl.cells[0]
    sph = pw.Sphere(c.L, c.N, c.ecut)
    gs = pw.ground_state_dense(sph, c.vloc, c.n_occ)
    s_ref, g_ref, _ = gradient.grad_vloc(gs, wl.phi)
    cell = gw.Cell(c.L, c.N, c.ecut, c.vloc)
    cell.set_occupied(gs.C, gs.eps)
    s64, g64 = cell.grad_vloc(wl.phi, wl.k, gw.GW_FP64)
    s32, g32 = cell.grad_vloc(wl.phi, wl.k, gw.GW_MIXED)
    cell.close()
    assert abs(s64 - s_ref) < 1e-10 * abs(s_ref)
    assert rel(g64, g_ref) < 1e-8
    assert rel(g32, g_ref) < 1e-6


def test_gradient_with_deflation():
    """The adjoint's Sternheimer solves with a deflation block: same gradient."""
    c, sph, gs, phi = _case(W.small(), [1.0, 2.0, 3.0])
    s_ref, g_ref, _ = gradient.grad_vloc(gs, phi)
    e = gs.eps_all
    m = next(k for k in range(2, 12) if e[gs.n_occ + k] - e[gs.n_occ + k - 1] > 1e-3)
    cell = gw.Cell(c.L, c.N, c.ecut, c.vloc)
    cell.set_occupied(gs.C, gs.eps)
    cell.set_deflation(gs.C_all[gs.n_occ:gs.n_occ + m], e[gs.n_occ:gs.n_occ + m])
    s, g = cell.grad_vloc(phi, 30, gw.GW_FP64)
    cell.close()
    assert abs(s - s_ref) < 1e-9 * abs(s_ref)
    assert rel(g, g_ref) < 1e-9
