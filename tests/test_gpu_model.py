"""Parity of the model operator (Sec. Dielectric model, Eq. model_eq) and of
the two-basis split (Eq. subs_epsilon) on the GPU against the FP64 oracle.

The model path has no iterative solve: with GW_FP64 every step is FP64
arithmetic, so the applications agree with the oracle to rounding (1e-12
relative) and the Lanczos coefficients and the split to 1e-10.  GW_MIXED runs
the model in FP64 too (it has no solve whose FP64 residual could refine FP32
transforms), so the mixed results meet 1e-6 everywhere.
"""
import numpy as np
import pytest

import workloads as W
from oracle import lanczos, pw, response
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


def _case(wl):
    cell = wl.cells[0]
    sph = pw.Sphere(cell.L, cell.N, cell.ecut)
    gs = pw.ground_state_dense(sph, cell.vloc, cell.n_occ)
    return cell, sph, gs


@pytest.fixture(scope="module")
def tiny():
    return _case(W.tiny())


def _model_cell(cell, gs):
    c = gw.Cell(cell.L, cell.N, cell.ecut, cell.vloc, 0)
    c.set_occupied(gs.C, gs.eps)
    c.set_operator(gw.GW_OP_MODEL)
    return c


@pytest.mark.parametrize("omega", [0.0, 0.15, 0.2 + 0.1j])
def test_model_chi0_and_eps(tiny, omega):
    cell, sph, gs = tiny
    c = _model_cell(cell, gs)
    f = W.random_fields(301, 3, sph.ng)
    dn = c.apply_chi0(f, [omega], gw.GW_FP64)[0]
    D = response.Dielectric(gs, omega, route="model")
    for b in range(3):
        ref = response.chi0_model(gs, f[b], omega)
        assert rel(dn[b], ref if np.iscomplexobj(dn) else ref.real) < 1e-12
    out = c.apply_eps(f[:2], [omega], gw.GW_FP64)[0]
    out32 = c.apply_eps(f[:2], [omega], gw.GW_MIXED)[0]
    dn32 = c.apply_chi0(f, [omega], gw.GW_MIXED)[0]
    for b in range(2):
        ref = D.apply(f[b])
        assert rel(out[b], ref) < 1e-12
        assert rel(out32[b], ref) < 1e-6
        assert rel(dn32[b], response.chi0_model(gs, f[b], omega)) < 1e-6
    c.close()


def test_model_complex_fields(tiny):
    cell, sph, gs = tiny
    c = _model_cell(cell, gs)
    x = W.random_fields(302, 2, sph.ng, complex_=True)
    omegas = [0.1, 0.3 + 0.2j]
    out = c.apply_eps(x, omegas, gw.GW_FP64)
    for o, om in enumerate(omegas):
        D = response.Dielectric(gs, om, route="model")
        for b in range(2):
            assert rel(out[o, b], D.apply(x[b], real=False)) < 1e-12
    c.close()


@pytest.mark.parametrize("seed_idx,N,L,ecut,n_occ", [(10, 12, 8.0, 3.0, 2), (12, 15, 7.5, 3.5, 5),
                                                    (14, 18, 9.0, 4.0, 6)])
def test_model_chi0_ragged_cells(seed_idx, N, L, ecut, n_occ):
    """Other grids (15^3: radix 3 and 5) and occupied counts."""
    cell, sph, gs = _case(W.small(N=N, L=L, ecut=ecut, n_occ=n_occ, n_wells=3, seed_idx=seed_idx))
    c = _model_cell(cell, gs)
    f = W.random_fields(303, 5, sph.ng)
    dn = c.apply_chi0(f, [0.0, 0.4], gw.GW_FP64)
    for o, om in enumerate([0.0, 0.4]):
        for b in range(5):
            assert rel(dn[o, b], response.chi0_model(gs, f[b], om).real) < 1e-12
    c.close()


@pytest.mark.parametrize("V0,omega", [(-0.37, 0.0), (-0.37, 0.05), (0.21, 0.1 + 0.2j)])
def test_model_constant_potential_closed_form_gpu(V0, omega):
    """Plane-wave occupied state (V_loc = V0, e_0 = V0): the model is diagonal in
    G, P~(G) = -(2/Omega) [1/(|G|^2/2 - V0 - omega) + 1/(|G|^2/2 - V0 + omega)]
    for G != 0 in the sphere; checked without the oracle's model code."""
    L, N, ecut = 8.0, 12, 3.0
    sph = pw.Sphere(L, N, ecut)
    c = gw.Cell(L, N, ecut, np.full(sph.ng, V0), 0)
    c.set_occupied(np.ones((1, 1)) * (sph.miller == 0).all(axis=1)[None, :], [V0])
    c.set_operator(gw.GW_OP_MODEL)
    f = W.random_fields(304, 1, sph.ng, complex_=True)
    dn = c.apply_chi0(f, [omega], gw.GW_FP64)[0, 0]
    G2 = sph.gvec_norm() ** 2
    insph = np.zeros(sph.ng, bool)
    insph[sph.index] = True
    m = insph & (G2 > 0)
    expect = np.zeros(sph.ng, complex)
    t = G2[m] / 2 - V0
    expect[m] = -(2.0 / sph.omega_vol) * (1.0 / (t - omega) + 1.0 / (t + omega))
    assert rel(sph.fwd(dn), expect * sph.fwd(f[0])) < 1e-12
    c.close()


def test_model_lanczos(tiny):
    wl = W.tiny()
    cell, sph, gs = tiny
    c = _model_cell(cell, gs)
    x0 = wl.starts[0][0]
    K = 20
    w = sph.omega_vol / sph.ng
    D = response.Dielectric(gs, 0.0, route="model")
    ar, br, _ = lanczos.lanczos(lambda x: D.apply(x), x0, K, weight=w)
    a, b, Q = c.lanczos(x0, K, 0.0, gw.GW_FP64, basis=True)
    assert rel(a, ar) < 1e-10 and rel(b, br) < 1e-10
    assert np.abs(w * Q @ Q.T - np.eye(K)).max() < 1e-12
    # the mixed precision runs the model operator in FP64 (no solve whose
    # residual could refine FP32 transforms): the mixed path's 1e-6 holds
    a32, b32, _ = c.lanczos(x0, K, 0.0, gw.GW_MIXED)
    assert rel(a32, ar) < 1e-6 and rel(b32, br) < 1e-6
    c.close()


def test_model_block_lanczos_complex(tiny):
    wl = W.tiny()
    cell, sph, gs = tiny
    c = _model_cell(cell, gs)
    X0 = W.random_fields(305, 2, sph.ng)
    omega = 0.25 + 0.1j
    w = sph.omega_vol / sph.ng
    D = response.Dielectric(gs, omega, route="model")
    Ar, Br, _ = lanczos.block_lanczos(lambda X: np.array([D.apply(x, real=False) for x in X]),
                                      X0.astype(complex), 3, weight=w, bilinear=True)
    A, B, _ = c.block_lanczos(X0, 3, omega, gw.GW_FP64)
    assert rel(np.array(A), np.array(Ar)) < 1e-10
    assert rel(np.array(B), np.array(Br)) < 1e-10
    c.close()


def test_epsinv_split(tiny):
    """Eq. subs_epsilon from a 6-step Sternheimer basis and a 20-step model
    basis, for the common start field and a second field (m = 2); the oracle
    builds its own bases and M."""
    wl = W.tiny()
    cell, sph, gs = tiny
    w = sph.omega_vol / sph.ng
    x0 = wl.starts[0][0]
    phi = np.stack([x0, W.random_fields(306, 1, sph.ng)[0]])
    k, km = 6, 20
    D = response.Dielectric(gs, 0.0, route="sos")
    Dm = response.Dielectric(gs, 0.0, route="model")
    ar, br, Qr = lanczos.lanczos(lambda x: D.apply(x), x0, k, weight=w)
    amr, bmr, Qmr = lanczos.lanczos(lambda x: Dm.apply(x), x0, km, weight=w)
    Qr, Qmr = np.array(Qr), np.array(Qmr)
    M = lanczos.compress(lambda x: Dm.apply(x), Qr, w).real
    ref = lanczos.epsinv_split(w * phi @ Qr.T, lanczos.tridiag(ar, br), M, w * phi @ Qmr.T,
                               lanczos.tridiag(amr, bmr))
    c = gw.Cell(cell.L, cell.N, cell.ecut, cell.vloc, 0)
    c.set_occupied(gs.C, gs.eps)
    lz = c.lanczos(x0, k, 0.0, gw.GW_FP64, basis=True)
    c.set_operator(gw.GW_OP_MODEL)
    lzm = c.lanczos(x0, km, 0.0, gw.GW_FP64, basis=True)
    c.set_operator(gw.GW_OP_STERNHEIMER)
    got = c.epsinv_split(phi, lz, lzm, 0.0)
    assert rel(got, ref) < 1e-10
    # the split is a different estimate from either single basis
    plain = (w * x0 @ x0) * (np.linalg.inv(lanczos.tridiag(ar, br))[0, 0] - 1.0)
    assert abs(got[0, 0] - plain) > 1e-8 * abs(plain)
    c.close()


def test_operator_switch_and_errors(tiny):
    cell, sph, gs = tiny
    c = gw.Cell(cell.L, cell.N, cell.ecut, cell.vloc, 0)
    c.set_occupied(gs.C, gs.eps)
    f = W.random_fields(307, 1, sph.ng)
    exact = c.apply_chi0(f, [0.0], gw.GW_FP64)[0, 0]
    c.set_operator(gw.GW_OP_MODEL)
    with pytest.raises(gw.GwError) as e:
        c.grad_vloc(f[0], 2)
    assert e.value.status == 8
    model = c.apply_chi0(f, [0.0], gw.GW_FP64)[0, 0]
    assert rel(model, exact) > 1e-3
    c.set_operator(gw.GW_OP_STERNHEIMER)
    assert rel(c.apply_chi0(f, [0.0], gw.GW_FP64)[0, 0], exact) < 1e-12
    with pytest.raises(gw.GwError) as e:
        c.set_operator(2)
    assert e.value.status == 1
    with pytest.raises(gw.GwError) as e:
        gw.gw_epsinv_split(c.ctx, f, np.zeros((3, sph.ng)), np.ones(3), np.ones(2), np.zeros((1, sph.ng)),
                           np.ones(1), np.ones(1), float("nan"), np.zeros((1, 1)))
    assert e.value.status == 7
    c.close()
