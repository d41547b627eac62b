"""Parity of the CUDA path (through the C ABI) against the FP64 oracle.

Tolerances: FP64 path <= 1e-10 relative (alpha, beta, eps^-1 elements; the
operator applications themselves to ~1e-12); mixed path <= 1e-6.
"""
import numpy as np
import pytest

import workloads as W
from oracle import coulomb, lanczos, pw, response
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


def make(cell, gs=None, coulomb_kind=0):
    c = gw.Cell(cell.L, cell.N, cell.ecut, cell.vloc, coulomb_kind)
    if gs is not None:
        c.set_occupied(gs.C, gs.eps)
    return c


# ---------------------------------------------------------------------------
def test_sphere_bit_exact():
    for cell in [W.tiny().cells[0], W.small().cells[0], W.molecule().cells[0],
                 W.differentiation().cells[0], W.small(N=45, L=14.0, ecut=4.0).cells[0],
                 W.small(N=30, L=12.0, ecut=5.0).cells[0]]:
        sph = pw.Sphere(cell.L, cell.N, cell.ecut)
        c = make(cell)
        assert c.npw == sph.npw
        assert np.array_equal(c.sphere(), sph.miller)
        c.close()


@pytest.mark.parametrize("N,L,ecut", [(16, 10.0, 5.0), (18, 9.0, 4.0), (45, 14.0, 4.0), (24, 11.0, 6.0)])
def test_apply_h(N, L, ecut):
    cell = W.small(N=N, L=L, ecut=ecut, n_wells=3).cells[0]
    sph = pw.Sphere(cell.L, cell.N, cell.ecut)
    c = make(cell)
    rng = np.random.default_rng(N)
    X = rng.standard_normal((5, sph.npw)) + 1j * rng.standard_normal((5, sph.npw))
    ref = pw.h_apply(sph, cell.vloc, X)
    assert rel(c.apply_h(X, gw.GW_FP64), ref) < 1e-13
    assert rel(c.apply_h(X, gw.GW_MIXED), ref) < 2e-6
    c.close()


@pytest.fixture(scope="module")
def tiny():
    wl = W.tiny()
    cell = wl.cells[0]
    sph = pw.Sphere(cell.L, cell.N, cell.ecut)
    gs = pw.ground_state_dense(sph, cell.vloc, cell.n_occ)
    return wl, cell, sph, gs


@pytest.mark.parametrize("omega", [0.0, 0.15])
def test_apply_chi0_fp64(tiny, omega):
    wl, cell, sph, gs = tiny
    c = make(cell, gs)
    f = W.random_fields(101, 3, sph.ng)
    out = c.apply_chi0(f, [omega], gw.GW_FP64)[0]
    for b in range(3):
        ref = response.chi0_sos(gs, f[b], omega).real
        assert rel(out[b], ref) < 1e-11
    st = c.stats()
    assert st["max_residual"] < 1e-12
    c.close()


def test_apply_eps_fp64_and_mixed(tiny):
    wl, cell, sph, gs = tiny
    c = make(cell, gs)
    D = response.Dielectric(gs, 0.0)
    f = W.random_fields(102, 2, sph.ng)
    out64 = c.apply_eps(f, [0.0], gw.GW_FP64)[0]
    out32 = c.apply_eps(f, [0.0], gw.GW_MIXED)[0]
    for b in range(2):
        ref = D.apply(f[b])
        assert rel(out64[b], ref) < 1e-12
        assert rel(out32[b], ref) < 1e-6
    c.close()


def test_lanczos_tiny_fp64(tiny):
    wl, cell, sph, gs = tiny
    c = make(cell, gs)
    D = response.Dielectric(gs, 0.0)
    wgt = sph.omega_vol / sph.ng
    x0 = wl.starts[0][0]
    a_ref, b_ref, Q_ref = lanczos.lanczos(D.apply, x0, wl.k, wgt)
    a, b, Q = c.lanczos(x0, wl.k, 0.0, gw.GW_FP64, basis=True)
    assert rel(a, a_ref) < 1e-10
    assert rel(b, b_ref) < 1e-10
    assert np.abs(wgt * Q @ Q.T - np.eye(wl.k)).max() < 1e-13
    Ti = c.epsinv(a, b)
    Ti_ref = lanczos.epsinv_lanczos(a_ref, b_ref)
    assert np.abs(Ti - Ti_ref).max() / np.abs(Ti_ref).max() < 1e-10
    c.close()


def test_lanczos_tiny_mixed(tiny):
    wl, cell, sph, gs = tiny
    c = make(cell, gs)
    D = response.Dielectric(gs, 0.0)
    wgt = sph.omega_vol / sph.ng
    x0 = wl.starts[0][0]
    a_ref, b_ref, _ = lanczos.lanczos(D.apply, x0, wl.k, wgt)
    a, b, _ = c.lanczos(x0, wl.k, 0.0, gw.GW_MIXED)
    assert rel(a, a_ref) < 1e-6
    assert rel(b, b_ref) < 1e-6
    Ti = c.epsinv(a, b)
    Ti_ref = lanczos.epsinv_lanczos(a_ref, b_ref)
    assert np.abs(Ti - Ti_ref).max() / np.abs(Ti_ref).max() < 1e-6
    c.close()


def test_epsinv_matches_dense_inverse():
    rng = np.random.default_rng(4)
    a = 1.5 + rng.random(37)
    b = 0.3 * rng.random(36)
    cell = W.tiny().cells[0]
    c = make(cell)
    Ti = c.epsinv(a, b)
    assert rel(Ti, np.linalg.inv(lanczos.tridiag(a, b))) < 1e-13
    c.close()


def test_free_electron_closed_form_gpu():
    """V = 0, one occupied state: chi0(G) = -(2/Omega)|G|^2/((|G|^2/2)^2 - w^2)."""
    cell = W.Cell(8.0, 12, 3.0, 1, np.zeros((0, 3)), 0.0, 1.0)
    sph = pw.Sphere(cell.L, cell.N, cell.ecut)
    gs = pw.ground_state_dense(sph, np.zeros(sph.ng), 1)
    c = make(cell, gs)
    f = W.random_fields(7, 1, sph.ng)
    for omega in (0.0, 0.1):
        dn = c.apply_chi0(f, [omega], gw.GW_FP64)[0, 0]
        G2 = sph.gvec_norm() ** 2
        insph = np.zeros(sph.ng, bool)
        insph[sph.index] = True
        expect = np.zeros(sph.ng)
        m = insph & (G2 > 0)
        expect[m] = -(2.0 / sph.omega_vol) * G2[m] / ((G2[m] / 2) ** 2 - omega ** 2)
        assert rel(sph.fwd(dn), expect * sph.fwd(f[0])) < 1e-12
    c.close()


def test_persistent_cg_matches_multi_launch(tiny):
    """The one-launch CG (the grid-wide cooperative kernel, or one cluster per
    column) and the multi-launch CG agree."""
    wl, cell, sph, gs = tiny
    f = W.random_fields(103, 2, sph.ng)
    outs = {}
    for kind in (gw.GW_CG_PERSISTENT, gw.GW_CG_CLUSTER, gw.GW_CG_MULTI_LAUNCH):
        c = make(cell, gs)
        c.set_cg_kernel(kind)
        outs[kind] = (c.apply_eps(f, [0.0], gw.GW_FP64), c.apply_eps(f, [0.0], gw.GW_MIXED))
        c.close()
    o1, o1m = outs[gw.GW_CG_PERSISTENT]
    for kind in (gw.GW_CG_CLUSTER, gw.GW_CG_MULTI_LAUNCH):
        o, om = outs[kind]
        assert rel(o1, o) < 1e-12
        assert rel(o1m, om) < 1e-8


def test_solver_iteration_cap_reports_noconv(tiny):
    """Sec. "Avoiding summations": a Sternheimer solve that does not reach its
    tolerance is a failure of the method; with one inner iteration per pass and
    two passes the library must say so (GW_E_NOCONV, status 4) and still write
    finite outputs, and the context must work normally afterwards."""
    wl, cell, sph, gs = tiny
    f = W.random_fields(104, 1, sph.ng)
    c = make(cell, gs)
    good = c.apply_eps(f, [0.0], gw.GW_FP64)
    c.set_solver(max_iter=1, max_outer=2)
    out = np.full((1, 1, sph.ng), np.nan)
    with pytest.raises(gw.GwError) as ei:
        gw.gw_apply_eps(c.ctx, np.ascontiguousarray(f), [0.0], out, gw.GW_FP64)
    assert ei.value.status == 4
    assert "did not converge" in gw.gw_last_error(c.ctx)
    assert np.all(np.isfinite(out))
    c.set_solver(max_iter=20000, max_outer=12)
    assert rel(c.apply_eps(f, [0.0], gw.GW_FP64), good) < 1e-12
    c.close()


@pytest.mark.parametrize("prec", [gw.GW_FP64, gw.GW_MIXED])
def test_persistent_wait_bound_reports_timeout(tiny, prec):
    """Every device wait of the persistent CG is bounded: with the bound cut to
    one poll the CTAs that arrive first give up, every CTA returns, and the
    call reports GW_E_TIMEOUT (status 6) instead of hanging; the context then
    solves normally with the default bound."""
    wl, cell, sph, gs = tiny
    f = W.random_fields(105, 2, sph.ng)
    c = make(cell, gs)
    good = c.apply_eps(f, [0.0], prec)
    c.set_cg_kernel(gw.GW_CG_PERSISTENT, 1)
    with pytest.raises(gw.GwError) as ei:
        c.apply_eps(f, [0.0], prec)
    assert ei.value.status == 6
    c.set_cg_kernel(gw.GW_CG_PERSISTENT, 1 << 24)
    assert rel(c.apply_eps(f, [0.0], prec), good) < (1e-12 if prec == gw.GW_FP64 else 1e-8)
    c.close()


@pytest.mark.parametrize("omega", [0.3 + 0.1j, 0.25j, 0.9, 1.7 + 0.05j])
def test_apply_chi0_complex_and_indefinite(tiny, omega):
    """Frequencies that need simplified QMR: complex, and real above the
    excitation gap (H - e_v - w indefinite on P_c)."""
    wl, cell, sph, gs = tiny
    # keep clear of transitions (eps~ has poles at w = e_c - e_v)
    dmin = np.min(np.abs(np.subtract.outer(gs.eps_all[gs.n_occ:], gs.eps).ravel() - abs(np.real(omega))))
    assert np.imag(omega) != 0 or dmin > 1e-3
    c = make(cell, gs)
    f = W.random_fields(104, 2, sph.ng)
    out = c.apply_chi0(f, [omega], gw.GW_FP64)[0]
    outm = c.apply_chi0(f, [omega], gw.GW_MIXED)[0]
    for b in range(2):
        ref = response.chi0_sos(gs, f[b], omega)
        if np.imag(omega) == 0:
            ref = ref.real
        assert rel(out[b], ref) < 1e-10
        assert rel(outm[b], ref) < 1e-6
    c.close()


def test_apply_eps_complex_fields(tiny):
    """Complex input fields at complex frequency (the bilinear Lanczos case)."""
    wl, cell, sph, gs = tiny
    c = make(cell, gs)
    om = 0.4 + 0.1j
    D = response.Dielectric(gs, om)
    f = W.random_fields(105, 2, sph.ng, complex_=True)
    out = c.apply_eps(f, [om], gw.GW_FP64)[0]
    for b in range(2):
        assert rel(out[b], D.apply(f[b], real=False)) < 1e-10
    c.close()


def test_free_electron_complex_frequency_gpu():
    cell = W.Cell(8.0, 12, 3.0, 1, np.zeros((0, 3)), 0.0, 1.0)
    sph = pw.Sphere(cell.L, cell.N, cell.ecut)
    gs = pw.ground_state_dense(sph, np.zeros(sph.ng), 1)
    c = make(cell, gs)
    f = W.random_fields(8, 1, sph.ng)
    omega = 0.1 + 0.2j
    dn = c.apply_chi0(f, [omega], gw.GW_FP64)[0, 0]
    G2 = sph.gvec_norm() ** 2
    insph = np.zeros(sph.ng, bool)
    insph[sph.index] = True
    expect = np.zeros(sph.ng, complex)
    m = insph & (G2 > 0)
    expect[m] = -(2.0 / sph.omega_vol) * G2[m] / ((G2[m] / 2) ** 2 - omega ** 2)
    assert rel(sph.fwd(dn), expect * sph.fwd(f[0])) < 1e-11
    c.close()


@pytest.mark.parametrize("blk,omega", [(3, 0.0), (1, 0.35 + 0.1j), (2, 0.6 + 0.15j)])
def test_block_lanczos(tiny, blk, omega):
    """Block (Hermitian, real omega) and complex-symmetric (bilinear, complex
    omega) Lanczos against the oracle's recursion; T^-1 against a dense inverse."""
    from oracle import lanczos as OL
    wl, cell, sph, gs = tiny
    wgt = sph.omega_vol / sph.ng
    D = response.Dielectric(gs, omega)
    X0 = W.random_fields(106, blk, sph.ng)
    bil = np.imag(omega) != 0
    K = 6
    A_ref, B_ref, Q_ref = OL.block_lanczos(lambda X: np.array([D.apply(x, real=False) for x in X]),
                                           X0.astype(complex), K, wgt, bilinear=bil)
    c = make(cell, gs)
    A, B, Q = c.block_lanczos(X0, K, omega, gw.GW_FP64, basis=True)
    assert rel(A, A_ref) < 1e-10
    assert rel(B, B_ref) < 1e-10
    G = wgt * (Q @ Q.T if bil else Q.conj() @ Q.T)
    assert np.abs(G - np.eye(K * blk)).max() < 1e-12
    Ti = c.epsinv_block(A, B, bil)
    T = OL.block_tridiag(A_ref, B_ref, bilinear=bil)
    assert rel(Ti, np.linalg.inv(T)) < 1e-10
    Am, Bm, _ = c.block_lanczos(X0, K, omega, gw.GW_MIXED)
    assert rel(Am, A_ref) < 1e-6 and rel(Bm, B_ref) < 1e-6
    c.close()


@pytest.mark.parametrize("omega", [0.0, 0.9, 0.3 + 0.1j])
def test_preconditioner_same_solution(tiny, omega):
    """The kinetic preconditioner changes the iteration count, not the answer:
    both settings match the sum over states; the preconditioned solves take
    fewer iterations."""
    wl, cell, sph, gs = tiny
    f = W.random_fields(107, 2, sph.ng)
    c = make(cell, gs)
    outs, its = [], []
    for kind in (0, 1):
        c.set_precond(kind)
        outs.append(c.apply_chi0(f, [omega], gw.GW_FP64)[0])
        its.append(c.stats()["mean_iter"])
    for b in range(2):
        ref = response.chi0_sos(gs, f[b], omega)
        if np.imag(omega) == 0:
            ref = ref.real
        assert rel(outs[0][b], ref) < 1e-10
        assert rel(outs[1][b], ref) < 1e-10
    assert its[1] < its[0]
    with pytest.raises(gw.GwError):
        c.set_precond(2)
    c.close()


@pytest.mark.parametrize("omega", [0.0, 0.9, 0.3 + 0.1j])
def test_deflation_same_solution(tiny, omega):
    """Deflating the lowest conduction states changes the iterations, not the
    answer (their components are added exactly): both match the sum over
    states, and the solves at omega = 0 need fewer iterations."""
    wl, cell, sph, gs = tiny
    m = 5                                     # a clean cut: eps_all[9] - eps_all[8] = 0.045 Ha
    D, eD = gs.C_all[gs.n_occ:gs.n_occ + m], gs.eps_all[gs.n_occ:gs.n_occ + m]
    f = W.random_fields(108, 2, sph.ng)
    c = make(cell, gs)
    ref = [response.chi0_sos(gs, f[b], omega) for b in range(2)]
    if np.imag(omega) == 0:
        ref = [r.real for r in ref]
    outs, its = [], []
    for use in (False, True):
        c.set_deflation(D if use else np.zeros((0, sph.npw)), eD if use else np.zeros(0))
        for prec, tol in ((gw.GW_FP64, 1e-10), (gw.GW_MIXED, 1e-6)):
            out = c.apply_chi0(f, [omega], prec)[0]
            for b in range(2):
                assert rel(out[b], ref[b]) < tol, (use, prec)
            if prec == gw.GW_FP64:
                its.append(c.stats()["mean_iter"])
    if omega == 0.0:
        assert its[1] < its[0]
    # Lanczos with the block set: the oracle's alpha, beta
    c.set_deflation(D, eD)
    D0 = response.Dielectric(gs, 0.0)
    a_ref, b_ref, _ = lanczos.lanczos(D0.apply, wl.starts[0][0], 8, sph.omega_vol / sph.ng)
    a, b, _ = c.lanczos(wl.starts[0][0], 8, 0.0, gw.GW_FP64)
    assert rel(a, a_ref) < 1e-10 and rel(b, b_ref) < 1e-10
    c.close()


def test_deflation_argument_checks(tiny):
    wl, cell, sph, gs = tiny
    c = make(cell)
    with pytest.raises(gw.GwError):          # no occupied states yet
        c.set_deflation(gs.C_all[4:6], gs.eps_all[4:6])
    c.set_occupied(gs.C, gs.eps)
    with pytest.raises(gw.GwError):          # below the highest occupied energy
        c.set_deflation(gs.C_all[2:4], gs.eps_all[2:4])
    c.close()


def test_sqmr_graph_replay_matches_direct_launches(tiny):
    """The simplified-QMR iterations replayed from one captured CUDA graph give
    the launch-by-launch results bit for bit in FP64 (same kernels, same order)."""
    wl, cell, sph, gs = tiny
    f = W.random_fields(106, 2, sph.ng)
    c = make(cell, gs)
    c.set_graphs(1)
    on = c.apply_chi0(f, [0.3 + 0.1j], gw.GW_FP64)
    assert c.stats()["graph_replays"] > 0
    c.set_graphs(0)
    off = c.apply_chi0(f, [0.3 + 0.1j], gw.GW_FP64)
    assert c.stats()["graph_replays"] == 0
    c.close()
    assert rel(on, off) < 1e-14


@pytest.mark.parametrize("prec,tol", [(gw.GW_FP64, 1e-10), (gw.GW_MIXED, 1e-6)])
def test_squared_route_at_imaginary_frequency(tiny, prec, tol):
    """Eq. P2+ on the GPU: at omega = i w the squared Hermitian system gives
    x^- + x^+ directly; chi0 through it equals the sum over states, and equals
    the SQMR pair route, in one call that also holds a static and a complex
    frequency (those keep Eq. P2)."""
    wl, cell, sph, gs = tiny
    f = W.random_fields(107, 2, sph.ng)
    om = [0.25j, 0.0, 0.7j, 0.3 + 0.1j]
    c = make(cell, gs)
    c.set_imaginary_route(gw.GW_IMAG_SQUARED)
    sq = c.apply_chi0(f, om, prec)
    c.set_imaginary_route(gw.GW_IMAG_SQMR)
    pair = c.apply_chi0(f, om, prec)
    c.close()
    for k, w in enumerate(om):
        for b in range(2):
            ref = response.chi0_sos(gs, f[b], w)
            assert rel(sq[k][b], ref) < tol
            assert rel(pair[k][b], ref) < tol
