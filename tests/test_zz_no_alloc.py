"""gw_epsinv_elements_noalloc: the allocation-free T_K^-1 for callers that
cannot allocate device memory where they need the inverse (their device memory
is held by another allocator, or a cudaMalloc and its implicit device
synchronisation is not acceptable there).  It must give the same matrix as
gw_epsinv_elements (which uses context-owned workspaces) and as a dense
inverse, on consecutive calls that share its fixed scratch array.  Collected
last so that a run stopping at the first failure has run every other test
already."""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

gw = pytest.importorskip("paper_1408_3036_gb300")
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1408_3036_gb300 import _build
    _build.build()
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _tridiag(k, seed):
    rng = np.random.default_rng(seed)
    a = 1.5 + rng.random(k)            # eps~ >= 1: diagonally dominant, positive definite
    b = 0.4 * rng.random(max(k - 1, 1))
    return a, b[:k - 1]


def _dense(a, b):
    return np.diag(a) + np.diag(b, 1) + np.diag(b, -1)


def _call(lib, a, b, k, stream=None):
    """The raw C entry on device copies of a, b; returns (status, out)."""
    dev = torch.device("cuda")
    da = torch.tensor(a, dtype=torch.float64, device=dev)
    db = torch.tensor(b if k > 1 else np.zeros(1), dtype=torch.float64, device=dev)
    out = torch.full((k, k), np.nan, dtype=torch.float64, device=dev)
    st = lib.gw_epsinv_elements_noalloc(ctypes.c_void_p(da.data_ptr()), ctypes.c_void_p(db.data_ptr()), k,
                                        ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(stream))
    torch.cuda.synchronize()
    return st, out.cpu().numpy()


def test_noalloc_matches_context_inverse_on_consecutive_calls():
    lib = gw.load()
    import workloads as W
    cell = W.tiny().cells[0]
    c = gw.Cell(cell.L, cell.N, cell.ecut, cell.vloc)
    stream = torch.cuda.current_stream().cuda_stream
    for k, seed in ((37, 1), (100, 2), (1, 3)):     # calls in a row, different sizes, k = 1 without beta use
        a, b = _tridiag(k, seed)
        ref = c.epsinv(a, b)                          # existing entry point
        dense = np.linalg.inv(_dense(a, b))
        st, got = _call(lib, a, b, k, stream)
        assert st == 0
        assert np.abs(got - ref).max() <= 1e-13 * np.abs(ref).max()
        assert np.abs(got - dense).max() <= 1e-13 * np.abs(dense).max()
    c.close()


def test_noalloc_largest_size_against_the_tridiagonal_product():
    """k = 4096, the scratch's limit: T X = I on sampled columns (a property
    that holds at any size) and symmetry, then a small call right after it
    that reuses the same scratch."""
    lib = gw.load()
    k = 4096
    a, b = _tridiag(k, 7)
    st, X = _call(lib, a, b, k)
    assert st == 0
    cols = np.random.default_rng(8).choice(k, 64, replace=False)
    for j in cols:
        x = X[:, j]
        tx = a * x
        tx[:-1] += b * x[1:]
        tx[1:] += b * x[:-1]
        e = np.zeros(k)
        e[j] = 1.0
        assert np.abs(tx - e).max() < 1e-13
        assert np.abs(X[j, :] - x).max() < 1e-13 * np.abs(x).max()
    a2, b2 = _tridiag(9, 9)
    st, got = _call(lib, a2, b2, 9)
    assert st == 0
    assert np.abs(got - np.linalg.inv(_dense(a2, b2))).max() < 1e-14


def test_noalloc_zero_pivot_then_recovers():
    """alpha_1 = 0 is a zero pivot: GW_E_BREAKDOWN (5); the zero-pivot flag
    lives in the shared scratch, and the next good call must report 0 and the
    right inverse."""
    lib = gw.load()
    a, b = _tridiag(12, 4)
    a_bad = a.copy()
    a_bad[0] = 0.0
    st, _ = _call(lib, a_bad, b, 12)
    assert st == 5
    st, got = _call(lib, a, b, 12)
    assert st == 0
    assert np.abs(got - np.linalg.inv(_dense(a, b))).max() < 1e-14


def test_noalloc_rejects_sizes_beyond_its_scratch():
    lib = gw.load()
    dev = torch.device("cuda")
    k = 4097
    da = torch.ones(k, dtype=torch.float64, device=dev)
    db = torch.zeros(k, dtype=torch.float64, device=dev)
    out = torch.empty(1, dtype=torch.float64, device=dev)
    st = lib.gw_epsinv_elements_noalloc(ctypes.c_void_p(da.data_ptr()), ctypes.c_void_p(db.data_ptr()), k,
                                        ctypes.c_void_p(out.data_ptr()), None)
    assert st == 1


def test_noalloc_binding_checks_buffers_before_the_call():
    """The binding refuses buffers the kernel would overrun (checked on the host,
    no launch happens)."""
    dev = torch.device("cuda")
    a = torch.ones(8, dtype=torch.float64, device=dev)
    b = torch.zeros(7, dtype=torch.float64, device=dev)
    out = torch.empty((8, 8), dtype=torch.float64, device=dev)
    with pytest.raises(ValueError):
        gw.gw_epsinv_elements_noalloc(a, b, 8, torch.empty(63, dtype=torch.float64, device=dev))
    with pytest.raises(ValueError):
        gw.gw_epsinv_elements_noalloc(a, None, 8, out)
    with pytest.raises(ValueError):
        gw.gw_epsinv_elements_noalloc(a.float(), b, 8, out)
    with pytest.raises(ValueError):
        gw.gw_epsinv_elements_noalloc(a, b.cpu(), 8, out)
    with pytest.raises(ValueError):
        gw.gw_epsinv_elements_noalloc(a, b[:6], 8, out)
    gw.gw_epsinv_elements_noalloc(a[:1], None, 1, out)       # k = 1 needs no beta
