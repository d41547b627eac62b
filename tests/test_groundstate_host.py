"""The block LOBPCG used to prepare occupied states converges to the lowest
eigenpairs (host run with the oracle's H application in place of the GPU's)."""
import numpy as np
import pytest

import workloads as W
from oracle import pw

torch = pytest.importorskip("torch")


def test_lobpcg_matches_dense():
    from paper_1408_3036_gb300.groundstate import lowest_states
    wl = W.tiny()
    c = wl.cells[0]
    sph = pw.Sphere(c.L, c.N, c.ecut)
    gs = pw.ground_state_dense(sph, c.vloc, c.n_occ)

    class Fake:
        npw = sph.npw
        L = c.L

        @staticmethod
        def sphere():
            return sph.miller

    def apply(Yt):
        return torch.tensor(pw.h_apply(sph, c.vloc, Yt.numpy()))

    eps, psi, res = lowest_states(Fake, c.n_occ, tol=1e-10, apply=apply, device="cpu")
    assert res < 1e-10
    assert np.abs(eps - gs.eps_all[:c.n_occ + 1]).max() < 1e-12
    P1 = gs.C.T @ gs.C.conj()
    P2 = psi.T @ psi.conj()
    assert np.abs(P1 - P2).max() < 1e-9


def test_levels_below_covers_the_window():
    """Every eigenvalue of H up to the window's top, starting from a block
    smaller than their number (the block grows), against dense eigenvalues."""
    from paper_1408_3036_gb300.groundstate import levels_below
    wl = W.tiny()
    c = wl.cells[0]
    sph = pw.Sphere(c.L, c.N, c.ecut)
    ev = np.linalg.eigvalsh(pw.dense_h(sph, c.vloc))

    class Fake:
        npw = sph.npw
        L = c.L

        @staticmethod
        def sphere():
            return sph.miller

    def apply(Yt):
        return torch.tensor(pw.h_apply(sph, c.vloc, Yt.numpy()))

    emax = ev[c.n_occ - 1] + 1.0
    lev = levels_below(Fake, emax, c.n_occ + 1, tol=1e-8, apply=apply, device="cpu")
    ref = ev[ev <= emax]
    assert len(lev) == len(ref) > c.n_occ + 1
    assert np.abs(lev - ref).max() < 1e-9
