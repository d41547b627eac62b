"""The model operator (Eq. model_eq), the residue term (Eq. pe) and the
recycled bases (Eq. recy_eq) on the full molecule workload (L = 20 bohr, 48^3
grid, 12053 plane waves, 16 occupied states), by properties that hold at any
size (the oracle cannot diagonalise this cell in test time):

  * the model operator is symmetric, and its FP32 path follows FP64 (to 1e-4
    of the response: 8 of the 16 occupied states lie above zero, where the
    kinetic denominators become small);
  * the recycled matrix at w = 0 equals the Gram matrix of direct eps~(0)
    applications (the static solutions lie in the recycled bases);
  * Sigma^P at delta = 0 for the highest occupied state is minus half its own
    pole element at w = 0 (Theta(0) = 1/2, no other pole), and the mixed path
    follows FP64;
  * Sigma^c of the highest occupied state in the first eight Lanczos vectors:
    the mixed path follows FP64 part by part, and its residue part equals the
    Sigma^P entry's.
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


@pytest.fixture(scope="module")
def molecule():
    import torch
    from paper_1408_3036_gb300.groundstate import lowest_states
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    wl = W.molecule()
    c = wl.cells[0]
    cell = gw.Cell(c.L, c.N, c.ecut, c.vloc, 0, stream.cuda_stream)
    eps, psi, res = lowest_states(cell, c.n_occ + 4, tol=1e-10)
    assert res < 1e-8 and eps[c.n_occ] - eps[c.n_occ - 1] > 1e-3
    cell.set_occupied(psi[:c.n_occ], eps[:c.n_occ])
    yield wl, c, cell, eps, psi
    cell.close()
    torch.cuda.set_stream(torch.cuda.default_stream())


def test_model_operator_full_size(molecule):
    wl, c, cell, eps, psi = molecule
    w = c.L ** 3 / c.N ** 3
    X = W.random_fields(81, 2, c.N ** 3)
    cell.set_operator(gw.GW_OP_MODEL)
    Y = cell.apply_eps(X, [0.0], gw.GW_FP64)[0]
    Y32 = cell.apply_eps(X, [0.0], gw.GW_MIXED)[0]
    cell.set_operator(gw.GW_OP_STERNHEIMER)
    a, b = w * np.dot(X[0], Y[1]), w * np.dot(Y[0], X[1])
    assert abs(a - b) < 1e-12 * max(abs(a), w * np.dot(X[0], Y[0]))
    # the response part eps~ - 1: FP32 rounding amplified by the small kinetic
    # denominators of this cell's unbound occupied states
    assert np.abs(Y32 - Y).max() < 1e-4 * np.abs(Y - X).max()


def test_recycle_static_equals_direct_full_size(molecule):
    wl, c, cell, eps, psi = molecule
    w = c.L ** 3 / c.N ** 3
    F = W.random_fields(82, 5, c.N ** 3)
    F /= np.sqrt(w * (F * F).sum(axis=1))[:, None]
    E, kept = cell.recycle_eps(F, [0.0, 1.0], prec=gw.GW_FP64)
    assert kept == 10
    D = cell.apply_eps(F, [0.0], gw.GW_FP64)[0]
    ref = w * F @ (D - F).T
    assert np.abs(E[0] - ref).max() < 1e-9 * np.abs(ref).max()
    assert (np.diag(E[1]) > 0).all() and (np.diag(E[1]) < np.diag(E[0])).all()


def test_sigma_p_full_size(molecule):
    wl, c, cell, eps, psi = molecule
    n = c.n_occ
    cand = psi[:n + 4]
    ce = eps[:n + 4]
    occ = np.array([1] * n + [0] * 4)
    e = n - 1
    tot, terms = cell.sigma_p(cand[e], ce[e], 0.0, cand, ce, occ, k=4, prec=gw.GW_FP64)
    nz = np.nonzero(terms)[0]
    assert list(nz) == [e]                          # only the state itself, at w = 0
    el, _ = cell.sigma_p(cand[e], ce[e], 0.0, cand[e:e + 1], ce[e:e + 1], [0], k=4, prec=gw.GW_FP64)
    assert abs(tot + el) < 1e-12 * abs(el)          # -1/2 (occupied) against +1/2 (conduction)
    tot32, _ = cell.sigma_p(cand[e], ce[e], 0.0, cand, ce, occ, k=4, prec=gw.GW_MIXED)
    assert abs(tot32 - tot) < 1e-6 * abs(tot)


def test_sigma_c_full_size(molecule):
    import torch
    wl, c, cell, eps, psi = molecule
    n = c.n_occ
    dev = torch.device("cuda")
    start = torch.tensor(wl.starts[0][0], dtype=torch.float64, device=dev)
    a = torch.empty(8, dtype=torch.float64, device=dev)
    b = torch.empty(8, dtype=torch.float64, device=dev)
    Q = torch.empty((8, c.N ** 3), dtype=torch.float64, device=dev)
    gw.gw_lanczos(cell.ctx, start, 8, 0.0, a, b, Q, gw.GW_FP64)
    F = Q.cpu().numpy()
    r64 = cell.sigma_c(n - 1, 0.0, F, alpha=1.0, n_freq=8, k_h=8, k_p=4, prec=gw.GW_FP64)
    r32 = cell.sigma_c(n - 1, 0.0, F, alpha=1.0, n_freq=8, k_h=8, k_p=4, prec=gw.GW_MIXED)
    scale = max(abs(r64[k]) for k in ("integral", "SA", "SP"))
    for k in ("total", "integral", "SA", "SP"):
        assert abs(r32[k] - r64[k]) < 1e-6 * scale, k
    sp, _ = cell.sigma_p(psi[n - 1], eps[n - 1], 0.0, psi[:n], eps[:n], np.ones(n, int), k=4, prec=gw.GW_FP64)
    assert abs(r64["SP"] - sp) < 1e-9 * abs(sp)
