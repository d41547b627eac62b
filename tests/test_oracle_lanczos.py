"""Pins for the oracle's Lanczos recursion and inverse in the Lanczos basis."""
import numpy as np
import pytest

import workloads as W
from oracle import lanczos, pw, response
from tests.conftest import rel


@pytest.fixture(scope="module")
def dense_case():
    wl = W.small(N=10, L=6.0, ecut=2.5, n_wells=2, n_occ=2)
    c = wl.cells[0]
    sph = pw.Sphere(c.L, c.N, c.ecut)
    gs = pw.ground_state_dense(sph, c.vloc, c.n_occ)
    D = response.Dielectric(gs, 0.0)
    E = D.dense().real
    E = 0.5 * (E + E.T)
    return wl, sph, gs, D, E


def test_orthonormal_and_tridiagonalises(dense_case):
    wl, sph, gs, D, E = dense_case
    wgt = sph.omega_vol / sph.ng
    x0 = wl.starts[0][0]
    K = 15
    a, b, Q = lanczos.lanczos(D.apply, x0, K, wgt)
    G = wgt * Q @ Q.T
    assert np.abs(G - np.eye(K)).max() < 1e-13
    T = wgt * Q @ (E @ Q.T)                  # Q^T eps Q in the weighted product
    assert np.abs(T - lanczos.tridiag(a, b)).max() < 1e-12
    # Ritz values lie inside the spectrum and interlace between steps
    lam = np.linalg.eigvalsh(E)
    prev = None
    for k in range(2, K + 1):
        th = np.linalg.eigvalsh(lanczos.tridiag(a[:k], b[:k - 1]))
        assert th.min() >= lam.min() - 1e-12 and th.max() <= lam.max() + 1e-12
        if prev is not None:
            assert np.all(th[:-1] <= prev + 1e-12) and np.all(prev <= th[1:] + 1e-12)
        prev = th


def test_without_reorthogonalisation_orthogonality_degrades(dense_case):
    """Sec. Lanczos: without the Gram-Schmidt step the vectors lose
    orthogonality; with it they stay orthonormal to machine precision."""
    wl, sph, gs, D, E = dense_case
    wgt = sph.omega_vol / sph.ng
    x0 = wl.starts[0][0]
    K = 30
    _, _, Q0 = lanczos.lanczos(lambda x: E @ x, x0, K, wgt, reorth=0)
    _, _, Q2 = lanczos.lanczos(lambda x: E @ x, x0, K, wgt, reorth=2)
    err0 = np.abs(wgt * Q0 @ Q0.T - np.eye(K)).max()
    err2 = np.abs(wgt * Q2 @ Q2.T - np.eye(K)).max()
    assert err2 < 1e-13
    assert err0 > 1e3 * err2


def test_gauss_quadrature_monotone(dense_case):
    """|phi|^2 (T_k^-1)_11 increases with k and stays below <phi|eps^-1|phi>
    (Gauss quadrature for a positive definite operator)."""
    wl, sph, gs, D, E = dense_case
    wgt = sph.omega_vol / sph.ng
    phi = W.gaussian_phi(sph.L, sph.N, [1.0, 2.0, 2.5])
    s_true = wgt * phi @ np.linalg.solve(E, phi)
    a, b, _ = lanczos.lanczos(lambda x: E @ x, phi, 25, wgt)
    nrm2 = wgt * phi @ phi
    sk = [lanczos.quad_s(a[:k], b[:k - 1], nrm2) for k in range(1, 26)]
    assert np.all(np.diff(sk) >= -1e-13 * s_true)
    assert np.all(np.array(sk) <= s_true * (1 + 1e-13))
    assert abs(sk[-1] - s_true) < 1e-10 * s_true


def test_invariant_subspace_inverse_exact(dense_case):
    """Once the Krylov space is invariant (beta ~ 0), T^-1 = Q^T eps^-1 Q."""
    wl, sph, gs, D, E = dense_case
    wgt = sph.omega_vol / sph.ng
    x0 = wl.starts[0][0]
    a, b, Q = lanczos.lanczos(lambda x: E @ x, x0, 200, wgt)
    k = int(np.argmax(b < 1e-9 * np.abs(a).max())) + 1 if np.any(b < 1e-9 * np.abs(a).max()) else None
    if k is None:
        pytest.skip("no invariant subspace reached")
    Ti = lanczos.epsinv_lanczos(a[:k], b[:k - 1])
    Qk = Q[:k]
    ref = wgt * Qk @ np.linalg.solve(E, Qk.T)
    assert np.abs(Ti - ref).max() < 1e-10


def test_block_lanczos(dense_case):
    wl, sph, gs, D, E = dense_case
    wgt = sph.omega_vol / sph.ng
    X0 = W.random_fields(77, 3, sph.ng)
    A, B, Q = lanczos.block_lanczos(lambda X: X @ E.T, X0, 6, wgt)
    n = Q.shape[0]
    assert np.abs(wgt * Q @ Q.T - np.eye(n)).max() < 1e-13
    T = wgt * Q @ E @ Q.T
    assert np.abs(T - lanczos.block_tridiag(A, B)).max() < 1e-12
    # block 1 reduces to the single-vector recursion
    a1, b1, _ = lanczos.lanczos(lambda x: E @ x, X0[0], 6, wgt)
    A1, B1, _ = lanczos.block_lanczos(lambda X: X @ E.T, X0[:1], 6, wgt)
    assert np.abs(A1[:, 0, 0] - a1).max() < 1e-12
    assert np.abs(B1[:, 0, 0] - b1).max() < 1e-12


def test_complex_symmetric_lanczos(small_case):
    """Complex frequency: eps~ is complex symmetric; the bilinear-form Lanczos
    gives Q^T Q = I and Q^T eps Q = T."""
    _, c, sph, gs = small_case
    wgt = sph.omega_vol / sph.ng
    D = response.Dielectric(gs, 0.3 + 0.1j)
    x0 = W.random_fields(5, 1, sph.ng)[0].astype(complex)
    K = 6
    a, b, Q = lanczos.lanczos(lambda x: D.apply(x, real=False), x0, K, wgt, bilinear=True)
    assert np.abs(wgt * Q @ Q.T - np.eye(K)).max() < 1e-12
    AQ = np.array([D.apply(q, real=False) for q in Q])
    assert np.abs(wgt * Q @ AQ.T - lanczos.tridiag(a, b)).max() < 1e-12
