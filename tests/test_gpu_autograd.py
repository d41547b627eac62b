"""torch.autograd.Function for s = <phi|eps~^-1(0)|phi> (differentiation
configuration: L = 14 bohr, 32^3 grid, 8 Ha, 6 wells, N_occ = 8, K = 40).

The gradient that backward() leaves on V_loc is checked against the oracle's
gradient (itself pinned by central differences, tests/test_oracle_gradient.py)
and against central differences of the Function's own forward pass
(h = 1e-4 along a smooth direction).  The forward pass keeps only the Lanczos
basis; the first-order orbitals are recomputed in backward.
"""
import numpy as np
import pytest

import workloads as W
from oracle import gradient, pw
from tests.conftest import rel

pytestmark = pytest.mark.gpu
gw = pytest.importorskip("paper_1408_3036_gb300")
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1408_3036_gb300 import _build
    _build.build()
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


@pytest.fixture(scope="module")
def case():
    wl = W.differentiation()
    c = wl.cells[0]
    sph = pw.Sphere(c.L, c.N, c.ecut)
    gs = pw.ground_state_dense(sph, c.vloc, c.n_occ)
    s_ref, g_ref, _ = gradient.grad_vloc(gs, wl.phi)
    return wl, c, sph, s_ref, g_ref


def _s(wl, c, v, prec, grad=False):
    from paper_1408_3036_gb300.autograd import EpsInvQuad
    dev = torch.device("cuda")
    vt = torch.tensor(v, dtype=torch.float64, device=dev, requires_grad=grad)
    phi = torch.tensor(wl.phi, dtype=torch.float64, device=dev)
    s = EpsInvQuad.apply(vt, phi, c.L, c.ecut, c.n_occ, wl.k, prec)
    if grad:
        s.backward()
        return float(s), vt.grad.cpu().numpy()
    return float(s)


@pytest.mark.parametrize("prec,tol", [(0, 1e-7), (1, 1e-6)])
def test_autograd_gradient_matches_oracle(case, prec, tol):
    wl, c, sph, s_ref, g_ref = case
    s, g = _s(wl, c, c.vloc, prec, grad=True)
    assert abs(s - s_ref) < tol * abs(s_ref)
    assert rel(g, g_ref) < tol
    from paper_1408_3036_gb300.autograd import checkpoint_bytes, orbital_bytes
    print(f"checkpoint kept between passes: {checkpoint_bytes(c.N, wl.k) / 1e6:.2f} MB (Lanczos basis); "
          f"orbitals recomputed in backward instead of kept: {orbital_bytes(c.N, sph.npw, c.n_occ) / 1e6:.2f} MB")


def test_autograd_gradient_matches_central_differences(case):
    wl, c, sph, s_ref, g_ref = case
    _, g = _s(wl, c, c.vloc, 0, grad=True)
    L, N = c.L, c.N
    x = np.arange(N) * (L / N)
    X, Y, Z = np.meshgrid(x, x, x, indexing="ij")
    d = np.exp(-((X - 4.0) ** 2 + (Y - 7.0) ** 2 + (Z - 9.0) ** 2) / (2 * 1.2 ** 2)).reshape(-1)
    h = 1e-4
    fd = (_s(wl, c, c.vloc + h * d, 0) - _s(wl, c, c.vloc - h * d, 0)) / (2 * h)
    an = float(np.dot(g, d))
    assert abs(fd - an) < 1e-6 * abs(an)
