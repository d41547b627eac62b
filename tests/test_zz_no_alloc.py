"""gw_epsinv_elements_noalloc: the allocation-free T_K^-1 for callers that
cannot allocate device memory where they need the inverse.  It must give the
same matrix as gw_epsinv_elements (which uses context-owned workspaces), on
consecutive calls that share its fixed scratch array.  Collected last so that a
run stopping at the first failure has run every other test already."""
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


def test_noalloc_matches_context_inverse_on_consecutive_calls():
    lib = gw.load()
    import workloads as W
    cell = W.tiny().cells[0]
    c = gw.Cell(cell.L, cell.N, cell.ecut, cell.vloc)
    dev = torch.device("cuda")
    stream = torch.cuda.current_stream().cuda_stream
    for k, seed in ((37, 1), (100, 2)):             # two calls in a row, different sizes
        a, b = _tridiag(k, seed)
        ref = c.epsinv(a, b)                          # existing entry point
        da = torch.tensor(a, device=dev)
        db = torch.tensor(b if k > 1 else np.zeros(1), device=dev)
        out = torch.empty((k, k), dtype=torch.float64, device=dev)
        st = lib.gw_epsinv_elements_noalloc(ctypes.c_void_p(da.data_ptr()), ctypes.c_void_p(db.data_ptr()),
                                            k, ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(stream))
        assert st == 0
        got = out.cpu().numpy()
        assert np.abs(got - ref).max() <= 1e-13 * np.abs(ref).max()
    c.close()


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
