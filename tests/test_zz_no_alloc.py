"""The allocation-free pivoted Cholesky entry point (tdh_pchol_noalloc) against tdh_pchol.

tdh_pchol_noalloc serves callers that may not allocate device memory: its scratch is a
static array inside the library, so it is limited to n <= 65536 and calls on one device must
not overlap.  This file is collected last so that, if it fails, a run stopping at the first
failure has already run every other test; it passes alone in a fresh process too.
"""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def tdh():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1604_07486_gb300 as m
    from paper_1604_07486_gb300 import build
    build.build()
    return m


def _call(fn, h, n, j0, tol, kmax):
    import torch
    u = torch.zeros((kmax, n), dtype=torch.float64, device="cuda")
    piv = torch.zeros(kmax, dtype=torch.int64, device="cuda")
    K = ctypes.c_int64(-1)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    rc = fn(ctypes.c_void_p(h.data_ptr()), n, j0, tol, kmax, ctypes.c_void_p(u.data_ptr()),
            ctypes.c_void_p(piv.data_ptr()), ctypes.byref(K), stream)
    torch.cuda.synchronize()
    return rc, K.value, u[: max(K.value, 0)].cpu().numpy(), piv[: max(K.value, 0)].cpu().numpy()


@pytest.mark.parametrize("kind,j0,n,tol", [("cheb2leg", 1, 65536, 1e-15), ("leg2cheb", 0, 5000, 1e-12)])
def test_noalloc_matches_allocating_entry(tdh, kind, j0, n, tol):
    """Two calls in a row through the C ABI give the factors tdh_pchol gives (same pivots,
    same rank, factors within the pivoted-Cholesky test tolerance), and the library's
    allocation counter does not move across them."""
    L = tdh.lib()
    _, h, _, _ = tdh.symbols(kind, n)
    kmax = 128
    rc, K, u_ref, p_ref = _call(L.tdh_pchol, h, n, j0, tol, kmax)
    assert rc == 0 and K >= 10
    scale = np.abs(u_ref).max()
    made = tdh.alloc_stats()[0]  # device allocations the library has made so far
    for _ in range(2):
        rc, K2, u, p = _call(L.tdh_pchol_noalloc, h, n, j0, tol, kmax)
        assert rc == 0, L.tdh_last_error()
        assert K2 == K
        assert np.array_equal(p, p_ref)
        assert np.abs(u - u_ref).max() <= 1e-9 * scale
    assert tdh.alloc_stats()[0] == made  # the two calls allocated nothing


def test_noalloc_rejects_sizes_beyond_limit(tdh):
    import torch
    L = tdh.lib()
    n = 65537
    h = torch.ones(2 * n - 1, dtype=torch.float64, device="cuda")
    rc, K, _, _ = _call(L.tdh_pchol_noalloc, h, n, 0, 1e-12, 4)
    assert rc == -1
    assert b"65536" in L.tdh_last_error()
