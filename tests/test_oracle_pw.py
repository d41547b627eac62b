"""Pins for the oracle's plane-wave sphere, grid transforms and Hamiltonian."""
import math

import numpy as np
import pytest

from oracle import pw
from tests.conftest import rel


def test_sphere_count_brute_force():
    # |G|^2/2 <= ecut counted by a plain triple loop over integer vectors
    for L, N, ecut in [(10.0, 16, 5.0), (8.0, 12, 3.0), (14.0, 32, 8.0)]:
        sph = pw.Sphere(L, N, ecut)
        R = int(math.ceil(math.sqrt(2 * ecut) * L / (2 * math.pi))) + 1
        g = 2 * math.pi / L
        count = 0
        for a in range(-R, R + 1):
            for b in range(-R, R + 1):
                for c in range(-R, R + 1):
                    if 0.5 * (g * g) * (a * a + b * b + c * c) <= ecut:
                        count += 1
        assert sph.npw == count
        # canonical order = ascending linear grid index
        assert np.all(np.diff(sph.index) > 0)
        n = sph.miller % N
        assert np.array_equal((n[:, 0] * N + n[:, 1]) * N + n[:, 2], sph.index)


def test_h_matrix_element_index_order():
    # <G|V|G'> = Omega^-1 int e^{-iGr} V e^{iG'r} = V~(G - G').
    # V = A sin(2 pi x / L) has V~(+1,0,0) = A/(2i) and V~(-1,0,0) = -A/(2i).
    L, N, A = 8.0, 12, 0.7
    sph = pw.Sphere(L, N, 3.0)
    x = np.arange(N) * L / N
    X = np.meshgrid(x, x, x, indexing="ij")[0]
    v = (A * np.sin(2 * np.pi * X / L)).reshape(-1)
    H = pw.dense_h(sph, v)
    row = {tuple(m): i for i, m in enumerate(sph.miller)}
    i100, i000 = row[(1, 0, 0)], row[(0, 0, 0)]
    assert abs(H[i100, i000] - A / 2j) < 1e-14
    assert abs(H[i000, i100] + A / 2j) < 1e-14
    assert abs(H[i000, i000]) < 1e-14            # kinetic 0, no constant part
    assert np.allclose(H, H.conj().T, atol=1e-15)


def test_fft_h_matches_dense(small_case):
    _, c, sph, _ = small_case
    H = pw.dense_h(sph, c.vloc)
    rng = np.random.default_rng(5)
    X = rng.standard_normal((3, sph.npw)) + 1j * rng.standard_normal((3, sph.npw))
    assert rel(pw.h_apply(sph, c.vloc, X), X @ H.T) < 1e-13


def test_free_electron_spectrum():
    # V = 0: eigenvalues are |G|^2/2 over the sphere (closed form)
    sph = pw.Sphere(8.0, 12, 3.0)
    gs = pw.ground_state_dense(sph, np.zeros(sph.ng), 1)
    assert np.allclose(gs.eps_all, np.sort(sph.kin), atol=1e-13)
    # constant potential shifts every eigenvalue
    gs2 = pw.ground_state_dense(sph, np.full(sph.ng, -0.37), 1)
    assert np.allclose(gs2.eps_all, np.sort(sph.kin) - 0.37, atol=1e-13)


def test_eigenpairs(tiny_case):
    _, c, sph, gs = tiny_case
    r = pw.residuals(sph, c.vloc, gs.eps_all[:8], gs.C_all[:8])
    assert np.all(r ** 2 < 1e-24)
    assert np.abs(gs.C_all[:8].conj() @ gs.C_all[:8].T - np.eye(8)).max() < 1e-13
    # grid normalisation: <psi|psi> = (Omega/N_g) sum |Omega^-1/2 u|^2 = 1
    u = gs.u
    assert np.allclose(np.sum(np.abs(u) ** 2, axis=1) / sph.ng, 1.0, atol=1e-13)


def test_iterative_ground_state_matches_dense(small_case):
    _, c, sph, gs = small_case
    gsi, w, _ = pw.ground_state_iterative(sph, c.vloc, c.n_occ, tol=1e-10)
    assert np.abs(gsi.eps - gs.eps).max() < 1e-10
    # same occupied projector
    P1 = gs.C.T @ gs.C.conj()
    P2 = gsi.C.T @ gsi.C.conj()
    assert np.abs(P1 - P2).max() < 1e-8
