"""Parity of the correlation self-energy (Eq. e_c) on the GPU against the
oracle's evaluation in the same basis of fields (the first Lanczos vectors of
eps~(0)): the frequency integral, the Lorentzian analytic term and the residue
term separately.  Tolerances: FP64 1e-10, mixed 1e-6 (relative to the largest
part)."""
import numpy as np
import pytest

import workloads as W
from oracle import lanczos, pw, response, sigma_c as SC

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
    w = sph.omega_vol / sph.ng
    D = response.Dielectric(gs, 0.0)
    _, _, Q = lanczos.lanczos(lambda x: D.apply(x), wl.starts[0][0], 6, weight=w)
    return c, sph, gs, np.array(Q).real


@pytest.mark.parametrize("frac", [0.0, 0.3])
def test_sigma_c_parity(tiny, frac):
    c, sph, gs, F = tiny
    e = gs.n_occ - 1
    delta = frac * (gs.eps_all[gs.n_occ] - gs.eps_all[gs.n_occ - 1])
    ref, parts = SC.sigma_c_basis(gs, e, delta, 1.0, 8, F, k_h=6, k_p=4)
    cell = gw.Cell(c.L, c.N, c.ecut, c.vloc, 0)
    cell.set_occupied(gs.C, gs.eps)
    got = cell.sigma_c(e, delta, F, alpha=1.0, n_freq=8, k_h=6, k_p=4, prec=gw.GW_FP64)
    scale = max(abs(parts["integral"]), abs(parts["SA"]), abs(parts["SP"]), abs(ref))
    for k in ("integral", "SA", "SP"):
        assert abs(got[k] - parts[k]) < 1e-10 * scale, k
    assert abs(got["total"] - ref) < 1e-10 * scale
    assert (parts["SP"] != 0.0) == (frac == 0.0)
    got32 = cell.sigma_c(e, delta, F, alpha=1.0, n_freq=8, k_h=6, k_p=4, prec=gw.GW_MIXED)
    assert abs(got32["total"] - ref) < 1e-6 * scale
    cell.close()


def test_sigma_c_arguments(tiny):
    c, sph, gs, F = tiny
    cell = gw.Cell(c.L, c.N, c.ecut, c.vloc, 0)
    cell.set_occupied(gs.C, gs.eps)
    with pytest.raises(gw.GwError) as e:
        cell.sigma_c(gs.n_occ - 1, -0.05, F)              # below the highest occupied energy
    assert e.value.status == 8
    with pytest.raises(gw.GwError) as e:
        cell.sigma_c(gs.n_occ, 0.0, F)                    # not an occupied state
    assert e.value.status == 1
    with pytest.raises(gw.GwError) as e:
        cell.sigma_c(0, 1.0, F, alpha=0.0)
    assert e.value.status == 1
    cell.close()
