"""Projector coefficients on the tensor cores (tcgen05, TF32 hi/lo split, FP32
accumulation) against the CUDA-core dots and an FP64 reference.

The coefficients <C_v|y> depend on the library's choice of occupied basis (it
makes the states real in real space), so the FP64 check uses what does not:
sum_v |<C_v|y_j>|^2 = |P_v y_j|^2 for every column, from the oracle's own
occupied states.  Kernel 1 (tensor cores) and kernel 0 (CUDA cores) are
compared entry by entry.  Column counts span several 128-column tiles and a
ragged last tile; the sphere sizes are odd (8-byte row alignment)."""
import numpy as np
import pytest

import workloads as W
from oracle import pw

pytestmark = pytest.mark.gpu
gw = pytest.importorskip("paper_1408_3036_gb300")
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1408_3036_gb300 import _build
    _build.build()
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


@pytest.mark.parametrize("name,ncol", [("tiny", 300), ("slice", 1024), ("slice", 77)])
def test_tensor_core_projector_coefficients(name, ncol):
    wl = W.tiny() if name == "tiny" else W.block_freq_slice()
    c = wl.cells[0]
    sph = pw.Sphere(c.L, c.N, c.ecut)
    gs = pw.ground_state_dense(sph, c.vloc, c.n_occ)
    cell = gw.Cell(c.L, c.N, c.ecut, c.vloc)
    cell.set_occupied(gs.C, gs.eps)
    rng = np.random.default_rng(ncol)
    y = (rng.standard_normal((ncol, sph.npw)) + 1j * rng.standard_normal((ncol, sph.npw))).astype(np.complex64)
    dev = torch.device("cuda")
    ty = torch.tensor(y, device=dev)
    c0 = torch.empty((c.n_occ, ncol), dtype=torch.complex128, device=dev)
    c1 = torch.empty((c.n_occ, ncol), dtype=torch.complex128, device=dev)
    gw.gw_proj_coef(cell.ctx, ty, c0, 0)
    gw.gw_proj_coef(cell.ctx, ty, c1, 1)
    a0, a1 = c0.cpu().numpy(), c1.cpu().numpy()
    cell.close()
    # the CUDA-core dots carry FP32 rounding (about 1e-7 of the largest
    # coefficient); the tensor cores about 2e-6 (measured: the FP32
    # accumulation in tensor memory, not the 2^-22 of the TF32 hi/lo split);
    # the FP64 invariant checks each of them
    scale = np.abs(a0).max()
    print(f"max |tensor - CUDA cores| / max |coef| = {np.abs(a1 - a0).max() / scale:.2e}")
    assert np.abs(a1 - a0).max() < 5e-6 * scale
    ref = (np.abs(np.conj(gs.C) @ y.astype(np.complex128).T) ** 2).sum(0)     # |P_v y_j|^2
    for a in (a0, a1):
        assert np.abs((np.abs(a) ** 2).sum(0) - ref).max() < 1e-5 * ref.max()


def test_tensor_cores_in_the_mixed_sqmr_solver():
    """The block complex-frequency slice (1024 SQMR columns, 64 occupied
    states): the mixed solves with the tensor-core coefficients equal those with
    the CUDA-core dots to the solver tolerance, and meet the FP64 result to
    1e-6 (the FP64 refinement decides)."""
    wl = W.block_freq_slice()
    c = wl.cells[0]
    sph = pw.Sphere(c.L, c.N, c.ecut)
    gs = pw.ground_state_dense(sph, c.vloc, c.n_occ)
    cell = gw.Cell(c.L, c.N, c.ecut, c.vloc)
    cell.set_occupied(gs.C, gs.eps)
    f = W.random_fields(108, 8, sph.ng)
    om = [complex(wl.omegas[0])]
    d64 = cell.apply_chi0(f, om, gw.GW_FP64)
    cell.set_tensor_cores(1)
    dtc = cell.apply_chi0(f, om, gw.GW_MIXED)
    it_tc = cell.stats()["mean_iter"]
    cell.set_tensor_cores(0)
    dcc = cell.apply_chi0(f, om, gw.GW_MIXED)
    it_cc = cell.stats()["mean_iter"]
    cell.close()
    s = np.abs(d64).max()
    assert np.abs(dtc - d64).max() < 1e-6 * s
    assert np.abs(dcc - d64).max() < 1e-6 * s
    # the coefficients' accuracy must not cost the solver iterations
    print(f"mean SQMR iterations: tensor cores {it_tc:.1f}, CUDA cores {it_cc:.1f}")
    assert it_tc <= 1.15 * it_cc
