"""The block, complex-frequency workload.

Reduced slice against the oracle (L = 16 bohr, 32^3, 5 Ha, 2109 plane waves,
the workload's 24 wells, 64 occupied states, blocks of 8, two frequencies
Re + 0.1i, two block steps): the oracle diagonalises the cell densely and
applies eps~ by the sum over all conduction states; A_k and B_k of the
bilinear block recursion (Sec. Lanczos, block form, reading 12) match to
1e-10 (FP64) and 1e-6 (mixed).  The GPU side runs the same launch shape as
the full workload: 64 states x 2 signs x 8 fields = 1024 SQMR columns.

At full size (L = 24 bohr, 64^3 grid,
15 Ha, 38401 plane waves, 64 occupied states, blocks of 8, omega = Re + 0.1i):
properties that hold at any size, since the oracle cannot diagonalise this
cell or run its Sternheimer route in test time.

  * the block Lanczos vectors are orthonormal in the bilinear form (to 1e-13),
  * every A_k is complex symmetric,
  * the mixed-precision recursion equals the FP64 one to 1e-6 (first block step).
"""
import numpy as np
import pytest

import workloads as W
from oracle import lanczos, pw, response

pytestmark = pytest.mark.gpu

gw = pytest.importorskip("paper_1408_3036_gb300")


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1408_3036_gb300 import _build
    _build.build()
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def test_block_frequency_workload_full_size():
    import torch
    from paper_1408_3036_gb300.groundstate import lowest_states
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    wl = W.block_freq()
    c = wl.cells[0]
    cell = gw.Cell(c.L, c.N, c.ecut, c.vloc, 0, stream.cuda_stream)
    assert cell.npw == 38401
    eps, psi, res = lowest_states(cell, c.n_occ, tol=1e-10)
    assert res < 1e-8 and eps[c.n_occ] - eps[c.n_occ - 1] > 1e-3
    cell.set_occupied(psi, eps[:c.n_occ])
    X0 = wl.starts[0]
    omega = complex(wl.omegas[0])
    assert omega.imag == 0.1 and X0.shape == (8, c.N ** 3)
    wgt = c.L ** 3 / c.N ** 3
    Am, Bm, Qm = cell.block_lanczos(X0, 2, omega, gw.GW_MIXED, basis=True)
    G = wgt * (Qm @ Qm.T)
    assert np.abs(G - np.eye(len(G))).max() < 1e-13
    for a in Am:
        assert np.abs(a - a.T).max() < 1e-10 * np.abs(a).max()
    A64, _, _ = cell.block_lanczos(X0, 1, omega, gw.GW_FP64)
    assert np.abs(Am[0] - A64[0]).max() / np.abs(A64[0]).max() < 1e-6
    cell.close()
    torch.cuda.set_stream(torch.cuda.default_stream())


@pytest.fixture(scope="module")
def freq_slice():
    wl = W.block_freq_slice()
    c = wl.cells[0]
    sph = pw.Sphere(c.L, c.N, c.ecut)
    gs = pw.ground_state_dense(sph, c.vloc, c.n_occ)
    assert gs.gap() > 1e-3
    wgt = sph.omega_vol / sph.ng
    X0 = wl.starts[0].astype(complex)
    ref = []
    for om in wl.omegas:
        D = response.Dielectric(gs, complex(om), route="sos")
        As, Bs, _ = lanczos.block_lanczos(lambda Xb: np.array([D.apply(x, real=False) for x in Xb]), X0, wl.k,
                                          weight=wgt, bilinear=True)
        ref.append((np.array(As), np.array(Bs)))
    return wl, c, gs, ref


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-10), ("mixed", 1e-6)])
def test_block_frequency_slice_matches_oracle(freq_slice, prec, tol):
    wl, c, gs, ref = freq_slice
    cell = gw.Cell(c.L, c.N, c.ecut, c.vloc)
    cell.set_occupied(gs.C, gs.eps)
    p = gw.GW_FP64 if prec == "fp64" else gw.GW_MIXED
    for om, (Ar, Br) in zip(wl.omegas, ref):
        A, B, _ = cell.block_lanczos(wl.starts[0], wl.k, complex(om), p)
        assert np.abs(A - Ar).max() / np.abs(Ar).max() < tol
        assert np.abs(B[:wl.k - 1] - Br).max() / np.abs(Br).max() < tol
    st = cell.stats()
    assert st["columns"] >= 1024
    cell.close()
