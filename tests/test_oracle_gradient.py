"""Pins for the oracle's derivative of <phi|eps~^-1(0)|phi> w.r.t. V_loc."""
import numpy as np

import workloads as W
from oracle import gradient, lanczos, pw, response


def test_gradient_matches_central_differences(small_case):
    wl, c, sph, gs = small_case
    phi = W.gaussian_phi(c.L, c.N, [1.0, 2.0, 3.0])
    s, g, _ = gradient.grad_vloc(gs, phi)
    rng = np.random.default_rng(3)
    pts = rng.choice(sph.ng, 6, replace=False)
    dirs = rng.standard_normal((2, sph.ng))
    fp, fd = gradient.fd_grad(c.L, c.N, c.ecut, c.vloc, c.n_occ, phi, pts, dirs, h=1e-4)
    assert np.abs(fp - g[pts]).max() < 1e-6 * np.abs(g).max()
    assert np.abs(fd - dirs @ g).max() < 1e-6 * np.abs(dirs @ g).max()


def test_gradient_sums_to_zero(small_case):
    """A constant shift of V_loc leaves s unchanged."""
    wl, c, sph, gs = small_case
    phi = W.gaussian_phi(c.L, c.N, [2.0, 2.0, 2.0])
    _, g, _ = gradient.grad_vloc(gs, phi)
    assert abs(g.sum()) < 1e-12 * np.abs(g).sum()


def test_lanczos_s_matches_exact(small_case):
    wl, c, sph, gs = small_case
    phi = W.gaussian_phi(c.L, c.N, [1.0, 2.0, 3.0])
    s, u = gradient.s_exact(gs, phi)
    D = response.Dielectric(gs, 0.0)
    wgt = sph.omega_vol / sph.ng
    a, b, Q = lanczos.lanczos(D.apply, phi, 30, wgt)
    sK = lanczos.quad_s(a, b, wgt * phi @ phi)
    assert abs(sK - s) < 1e-11 * s
