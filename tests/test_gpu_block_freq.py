"""The block, complex-frequency workload at full size (L = 24 bohr, 64^3 grid,
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
