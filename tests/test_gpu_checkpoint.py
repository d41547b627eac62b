"""Lanczos checkpoint/resume through the C ABI (gw_lanczos_resume): a
recursion run in segments, or resumed from its checkpoint file after an
interruption, gives the coefficients of the uninterrupted run and of the
oracle; a damaged state is refused with GW_E_ARG before any step."""
import numpy as np
import pytest

import workloads as W
from oracle import lanczos as OL
from oracle import pw, response
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
def tiny():
    wl = W.tiny()
    c = wl.cells[0]
    sph = pw.Sphere(c.L, c.N, c.ecut)
    gs = pw.ground_state_dense(sph, c.vloc, c.n_occ)
    x0 = wl.starts[0][0]
    a_ref, b_ref, _ = OL.lanczos(response.Dielectric(gs, 0.0).apply, x0, 14, sph.omega_vol / sph.ng)
    return wl, c, gs, x0, a_ref, b_ref


def _cell(c, gs):
    cell = gw.Cell(c.L, c.N, c.ecut, c.vloc)
    cell.set_occupied(gs.C, gs.eps)
    cell.set_autotune(0)
    return cell


@pytest.mark.parametrize("prec,tol", [(0, 1e-10), (1, 1e-6)])
def test_segmented_and_resumed_runs_match(tiny, tmp_path, prec, tol):
    wl, c, gs, x0, a_ref, b_ref = tiny
    cell = _cell(c, gs)
    a, b, _ = cell.lanczos(x0, 14, 0.0, prec)
    p = tmp_path / "lz.npz"
    a2, b2, Q2 = cell.lanczos_checkpointed(x0, 14, p, 5, 0.0, prec)
    assert rel(a2, a) < 1e-12 and rel(b2, b) < 1e-12
    assert rel(a2, a_ref) < tol and rel(b2, b_ref) < tol
    # an interrupted run: 7 steps checkpointed, then continued from the file
    cell.lanczos_checkpointed(x0, 7, p, 7, 0.0, prec)
    a3, b3, Q3 = cell.lanczos_from_checkpoint(p, 14, prec)
    assert rel(a3, a) < 1e-12 and rel(b3, b) < 1e-12
    wgt = c.L ** 3 / c.N ** 3
    assert np.abs(wgt * Q3 @ Q3.T - np.eye(14)).max() < 1e-12
    cell.close()


def test_damaged_state_is_refused(tiny, tmp_path):
    wl, c, gs, x0, _, _ = tiny
    cell = _cell(c, gs)
    a, b, Q = cell.lanczos(x0, 6, 0.0, gw.GW_FP64, basis=True)
    for damage in ("row", "nan_alpha", "zero_beta"):
        Qd, ad, bd = Q.copy(), a[:5].copy(), b[:5].copy()
        if damage == "row":
            Qd[2] *= 1.0 + 1e-6
        elif damage == "nan_alpha":
            ad[1] = np.nan
        else:
            bd[3] = 0.0
        with pytest.raises(gw.GwError) as e:
            cell.lanczos_resume(Qd, ad, bd, 10)
        assert e.value.status == 1, damage        # GW_E_ARG
    # the context is still usable after the refusals
    a2, b2, _ = cell.lanczos_resume(Q, a[:5], b[:5], 10)
    a1, b1, _ = cell.lanczos(x0, 10, 0.0, gw.GW_FP64)
    assert rel(a2, a1) < 1e-12 and rel(b2, b1) < 1e-12
    # a damaged file never reaches the library
    from paper_1408_3036_gb300.checkpoint import CheckpointError
    p = tmp_path / "lz.npz"
    cell.lanczos_checkpointed(x0, 6, p, 6)
    raw = bytearray(p.read_bytes())
    raw[len(raw) // 3] ^= 0x01
    p.write_bytes(bytes(raw))
    with pytest.raises(CheckpointError):
        cell.lanczos_from_checkpoint(p, 10)
    cell.close()
