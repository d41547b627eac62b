"""Batches of uneven cells run concurrently (gw_batch_*) against the oracle and
against the same cells run one at a time."""
import numpy as np
import pytest

import workloads as W
from oracle import lanczos as OL
from oracle import pw, response
from tests.conftest import rel

pytestmark = pytest.mark.gpu

gw = pytest.importorskip("paper_1408_3036_gb300")


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1408_3036_gb300 import _build
    _build.build()
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _ground_states(cells):
    out = []
    for c in cells:
        sph = pw.Sphere(c.L, c.N, c.ecut)
        out.append((sph, pw.ground_state_dense(sph, c.vloc, c.n_occ)))
    return out


def _pole_distance(gs, omega):
    tr = np.subtract.outer(gs.eps_all[gs.n_occ:], gs.eps).ravel()
    return np.abs(tr - abs(np.real(omega))).min()


def _clear_omegas(omegas, states, idx):
    """Per cell, re-draw a real frequency that lies within 1e-3 Ha of one of
    the cell's transitions (eps~ has a pole there); seeds base + config index
    + 1000 attempt + 100 cell + frequency.  Returns (n_cells, n_omega)."""
    out = np.tile(np.array(omegas, complex), (len(states), 1))
    for i, (_, gs) in enumerate(states):
        for w in range(out.shape[1]):
            attempt = 0
            while np.imag(out[i, w]) == 0 and _pole_distance(gs, out[i, w]) <= 1e-3:
                attempt += 1
                out[i, w] = W.redraw_omega(W.BASE_SEED + idx + 1000 * attempt + 100 * i + w, 0.0, 1.0)
    return out


def _make_batch(cells, states, workers=0):
    b = gw.Batch([(c.L, c.N, c.ecut, c.vloc) for c in cells], workers=workers)
    for i, (sph, gs) in enumerate(states):
        b.cell(i).set_occupied(gs.C, gs.eps)
    return b


def test_batch_small_parity():
    """Five uneven cells, K = 8, omega = 0, two real (one or both above the
    gap: simplified QMR) and one complex (bilinear recursion)."""
    wl = W.batch_small()
    states = _ground_states(wl.cells)
    for sph, gs in states:
        for om in wl.omegas:
            assert np.imag(om) != 0 or _pole_distance(gs, om) > 1e-3
    b = _make_batch(wl.cells, states)
    A, B = b.lanczos([s[0] for s in wl.starts], wl.k, wl.omegas, gw.GW_FP64)
    assert np.all(b.last_status == 0)
    Am, Bm = b.lanczos([s[0] for s in wl.starts], wl.k, wl.omegas, gw.GW_MIXED)
    for i, (c, (sph, gs)) in enumerate(zip(wl.cells, states)):
        wgt = sph.omega_vol / sph.ng
        x0 = wl.starts[i][0]
        for w, om in enumerate(wl.omegas):
            D = response.Dielectric(gs, om)
            if np.imag(om) == 0:
                a_ref, b_ref, _ = OL.lanczos(D.apply, x0, wl.k, wgt)
            else:
                Ar, Br, _ = OL.block_lanczos(lambda X: np.array([D.apply(x, real=False) for x in X]),
                                             x0[None, :].astype(complex), wl.k, wgt, bilinear=True)
                a_ref, b_ref = Ar[:, 0, 0], Br[:, 0, 0]
            assert rel(A[i, w], a_ref) < 1e-10, (i, om)
            assert rel(B[i, w], b_ref) < 1e-10, (i, om)
            assert rel(Am[i, w], a_ref) < 1e-6, (i, om)
            assert rel(Bm[i, w], b_ref) < 1e-6, (i, om)
    b.close()


def test_batch_uneven_full_size():
    """The many-cell workload at full size on its six smallest cells (N up to
    48, K = 40, four real frequencies per cell): concurrent batch == the cells run
    one at a time (smallest and largest cell); alpha_1 sampled against the
    oracle; eps~(omega) >= 1 below the gap (Ritz values of T); mixed == FP64
    to 1e-6."""
    wl = W.batch()
    npw = [pw.Sphere(c.L, c.N, c.ecut).npw for c in wl.cells]
    pick = list(np.argsort(npw, kind="stable")[:6])
    cells = [wl.cells[i] for i in pick]
    starts = [wl.starts[i][0] for i in pick]
    states = _ground_states(cells)
    omegas = _clear_omegas(wl.omegas, states, 3)
    b = _make_batch(cells, states, workers=6)
    A, B = b.lanczos(starts, wl.k, omegas, gw.GW_FP64)
    assert np.all(b.last_status == 0)
    assert np.abs(A.imag).max() == 0 and np.abs(B.imag).max() == 0
    n_below = 0
    for i, (c, (sph, gs)) in enumerate(zip(cells, states)):
        gap = np.min(np.subtract.outer(gs.eps_all[gs.n_occ:], gs.eps))
        for w, om in enumerate(omegas[i]):
            if om.real < gap:
                n_below += 1
                ritz = np.linalg.eigvalsh(OL.tridiag(A[i, w].real, B[i, w].real))
                assert ritz.min() > 1.0 - 1e-10
        if i not in (0, len(cells) - 1):      # one at a time: the smallest and the largest cell
            continue
        one = gw.Cell(c.L, c.N, c.ecut, c.vloc)
        one.set_occupied(gs.C, gs.eps)
        for w, om in enumerate(omegas[i]):
            a1, b1, _ = one.lanczos(starts[i], wl.k, om.real, gw.GW_FP64)
            assert rel(A[i, w].real, a1) < 1e-10
            assert rel(B[i, w].real, b1) < 1e-10
        one.close()
    assert n_below > 0
    # sampled output: alpha_1 = <q_1|eps~ q_1> of the smallest cell, by the oracle
    sph, gs = states[0]
    wgt = sph.omega_vol / sph.ng
    q1 = starts[0] / np.sqrt(wgt * starts[0] @ starts[0])
    for w, om in enumerate(omegas[0]):
        a1 = wgt * q1 @ response.Dielectric(gs, om).apply(q1)
        assert abs(A[0, w, 0].real - a1) / abs(a1) < 1e-10
    Am, Bm = b.lanczos(starts, wl.k, omegas, gw.GW_MIXED)
    assert rel(Am.real, A.real) < 1e-6 and rel(Bm.real, B.real) < 1e-6
    b.close()


def test_batch_errors_are_per_cell():
    """A cell without occupied states fails alone; the others still run."""
    wl = W.batch_small(n_cells=3)
    states = _ground_states(wl.cells)
    b = gw.Batch([(c.L, c.N, c.ecut, c.vloc) for c in wl.cells])
    for i in (0, 2):
        b.cell(i).set_occupied(states[i][1].C, states[i][1].eps)
    with pytest.raises(gw.GwError) as e:
        b.lanczos([s[0] for s in wl.starts], 4, [0.0])
    assert "cell 1" in str(e.value)
    assert b.last_status[1] != 0 and b.last_status[0] == 0 and b.last_status[2] == 0
    b.close()


def _spectrum_to(sph, vloc, emax):
    """Eigenvalues of the cell's H up to emax (dense, by the oracle's H)."""
    import scipy.linalg as sl
    return sl.eigvalsh(pw.dense_h(sph, vloc), subset_by_value=(-np.inf, emax))


def test_batch_all_32_cells():
    """The many-cell workload at full size, all 32 cells (K = 40, four real
    frequencies per cell, mixed precision, SQMR iterations replayed from CUDA
    graphs).  Occupied states come from the library's eigensolver; a frequency
    within 1e-3 Ha of one of the cell's transitions (dense spectrum of the
    oracle's H) is re-drawn for that cell.  Every cell converges;
    eps~(omega) >= 1 below the gap (Ritz values of T); alpha_1 of the two
    smallest cells is sampled against the oracle; the graph-free run of two
    cells gives the same coefficients."""
    import time
    from paper_1408_3036_gb300 import groundstate
    wl = W.batch()
    b = gw.Batch([(c.L, c.N, c.ecut, c.vloc) for c in wl.cells], workers=8)
    omegas = np.tile(np.array(wl.omegas, complex), (len(wl.cells), 1))
    gaps = []
    import torch
    for i, c in enumerate(wl.cells):
        # input preparation on a context of its own on torch's stream (a batch
        # cell's context works on the batch's stream)
        prep = gw.Cell(c.L, c.N, c.ecut, c.vloc, 0, torch.cuda.current_stream().cuda_stream)
        eps, psi, res = groundstate.lowest_states(prep, c.n_occ, tol=1e-10)
        prep.close()
        assert res < 1e-9, (i, res)
        b.cell(i).set_occupied(psi, eps[:c.n_occ])
        sph = pw.Sphere(c.L, c.N, c.ecut)
        ev = _spectrum_to(sph, c.vloc, eps[c.n_occ - 1] + 1.01)
        assert np.abs(ev[:c.n_occ] - eps[:c.n_occ]).max() < 1e-8, i
        tr = np.subtract.outer(ev[c.n_occ:], ev[:c.n_occ]).ravel()
        gaps.append(ev[c.n_occ] - ev[c.n_occ - 1])
        for w in range(omegas.shape[1]):
            attempt = 0
            while np.abs(tr - omegas[i, w].real).min() <= 1e-3:
                attempt += 1
                omegas[i, w] = W.redraw_omega(W.BASE_SEED + 3 + 1000 * attempt + 100 * i + w, 0.0, 1.0)
    starts = [s[0] for s in wl.starts]
    t0 = time.perf_counter()
    A, B = b.lanczos(starts, wl.k, omegas, gw.GW_MIXED)
    t_all = time.perf_counter() - t0
    assert np.all(b.last_status == 0)
    assert np.abs(A.imag).max() == 0 and np.abs(B.imag).max() == 0
    n_below = 0
    for i in range(len(wl.cells)):
        for w, om in enumerate(omegas[i]):
            if om.real < gaps[i]:
                n_below += 1
                ritz = np.linalg.eigvalsh(OL.tridiag(A[i, w].real, B[i, w].real))
                assert ritz.min() > 1.0 - 1e-6, (i, om)
    assert n_below > 0
    npw = [b.cell(i).npw for i in range(len(wl.cells))]
    small = list(np.argsort(npw, kind="stable")[:2])
    for i in small:
        c = wl.cells[i]
        sph = pw.Sphere(c.L, c.N, c.ecut)
        gs = pw.ground_state_dense(sph, c.vloc, c.n_occ)
        wgt = sph.omega_vol / sph.ng
        q1 = starts[i] / np.sqrt(wgt * starts[i] @ starts[i])
        for w, om in enumerate(omegas[i]):
            a1 = wgt * q1 @ response.Dielectric(gs, om).apply(q1)
            assert abs(A[i, w, 0].real - a1) / abs(a1) < 1e-6, (i, om)
    b.close()
    # the same two cells without graph replay
    sub = [wl.cells[i] for i in small]
    b2 = gw.Batch([(c.L, c.N, c.ecut, c.vloc) for c in sub], workers=2)
    for j, i in enumerate(small):
        c = wl.cells[i]
        prep = gw.Cell(c.L, c.N, c.ecut, c.vloc, 0, torch.cuda.current_stream().cuda_stream)
        eps, psi, _ = groundstate.lowest_states(prep, c.n_occ, tol=1e-10)
        prep.close()
        b2.cell(j).set_occupied(psi, eps[:c.n_occ])
        b2.cell(j).set_graphs(0)
    A2, B2 = b2.lanczos([starts[i] for i in small], wl.k, omegas[small], gw.GW_MIXED)
    b2.close()
    assert rel(A2.real, A[small].real) < 1e-6 and rel(B2.real, B[small].real) < 1e-6
    print(f"32 cells, K = {wl.k}, 4 frequencies, mixed: {t_all:.1f} s")
