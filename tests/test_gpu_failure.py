"""Failure detection without a GPU fault.

Allocation failures (tdh_test_fail_alloc): the library's every device allocation goes
through two functions (plan memory and execute scratch); the hook makes the k-th of them fail
on the host, as an out-of-memory cudaMalloc would.  Each entry point must then return
TDH_ERR_NOMEM with a message and give back everything it had allocated (tdh_alloc_stats
counts the blocks held).

Device waits (tdh_test_tc_stall): with the hook on, split-bfloat16 kernels issue no
tensor-core products, so the mbarrier each CTA waits on is never signalled; the wait gives up
after about a second, the kernel finishes normally and the host reads TIMEOUT from the plan's
status word.  Nothing traps, faults or hangs.
"""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

NOMEM = -3


@pytest.fixture(scope="module")
def tdh():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1604_07486_gb300 as m
    from paper_1604_07486_gb300 import build
    build.build()
    yield m
    m.inject_alloc_failure(0)


def _create(tdh, kind, n, prec, **kw):
    """Plan creation through the C ABI; returns (rc, handle)."""
    p = tdh._Params()
    for i, v in enumerate(kw.get("params", ())):
        p.p[i] = float(v)
    p.prec = tdh.PRECS[prec]
    p.flags = (tdh.FLAG_RAGGED if kw.get("ragged") else 0) | tdh.FLAG_TARGET
    h = ctypes.c_void_p()
    rc = tdh.lib().tdh_plan_create(tdh.KINDS[kind], n, ctypes.byref(p), kw.get("tol", 2.5e-6),
                                   ctypes.byref(h))
    return rc, h


@pytest.mark.parametrize("kind,n,prec,kw", [
    ("leg2cheb", 4096, "fp32", {"ragged": True}),
    ("jac2jac", 3000, "fp64", {"params": (1.5, 0.25, -0.5, -0.5), "tol": 5e-13}),
    ("ultra2ultra", 2048, "fp32", {"params": (0.25, 2.75)}),
], ids=["leg2cheb-ragged", "jacobi-chain", "ultra-case3"])
def test_plan_create_fails_cleanly_at_every_allocation(tdh, kind, n, prec, kw):
    import torch
    torch.cuda.synchronize()
    made0, live0, _ = tdh.alloc_stats()
    rc, h = _create(tdh, kind, n, prec, **kw)
    assert rc == 0, tdh.lib().tdh_last_error()
    made1, live1, _ = tdh.alloc_stats()
    allocs = made1 - made0
    assert allocs >= 6 and live1 > live0
    assert tdh.lib().tdh_plan_destroy(h) == 0
    assert tdh.alloc_stats()[1] == live0
    # every allocation of the creation in turn (all of them when few, else a spread)
    ks = range(1, allocs + 1) if allocs <= 40 else np.unique(np.linspace(1, allocs, 40).astype(int))
    for k in ks:
        tdh.inject_alloc_failure(int(k))
        rc, h = _create(tdh, kind, n, prec, **kw)
        msg = tdh.lib().tdh_last_error()
        tdh.inject_alloc_failure(0)
        assert rc == NOMEM, (k, rc, msg)
        assert b"injected" in msg, msg
        assert not h.value
        assert tdh.alloc_stats()[1] == live0, f"plan blocks leaked after failure at {k}"
    # and the library still works afterwards
    rc, h = _create(tdh, kind, n, prec, **kw)
    assert rc == 0
    tdh.lib().tdh_plan_destroy(h)


def test_execute_scratch_failure_returns_nomem(tdh):
    """Ragged and host-buffer executes take scratch; a failed scratch allocation is reported
    and nothing is left held; the next call succeeds."""
    import torch
    n = 4096
    plan = tdh.Plan("leg2cheb", n, prec="fp32", ragged=True)
    lens = np.array([n, 100, 2000, 0, 513])
    offs = torch.tensor(np.r_[0, np.cumsum(lens)], dtype=torch.int64, device="cuda")
    x = torch.randn(int(lens.sum()), dtype=torch.float32, device="cuda")
    y = torch.zeros_like(x)
    plan.execute_ragged(x, offs, out=y)
    torch.cuda.synchronize()
    ref = y.clone()
    _, live0, scr0 = tdh.alloc_stats()
    tdh.inject_alloc_failure(1)
    with pytest.raises(tdh.TdhError) as ei:
        plan.execute_ragged(x, offs, out=y)
    tdh.inject_alloc_failure(0)
    assert ei.value.code == NOMEM
    torch.cuda.synchronize()
    assert tdh.alloc_stats()[1:] == (live0, scr0)
    y.zero_()
    plan.execute_ragged(x, offs, out=y)
    torch.cuda.synchronize()
    assert torch.equal(y, ref)
    # host buffers: device staging is scratch too
    hx = torch.randn(8, n, dtype=torch.float32).pin_memory()
    hy = torch.empty_like(hx).pin_memory()
    tdh.inject_alloc_failure(1)
    with pytest.raises(tdh.TdhError) as ei:
        plan.execute(hx, out=hy)
    tdh.inject_alloc_failure(0)
    assert ei.value.code == NOMEM
    torch.cuda.synchronize()
    assert tdh.alloc_stats()[1:] == (live0, scr0)
    plan.close()


def test_pchol_allocation_failure(tdh):
    """tdh_pchol allocates its scratch; a failure there is NOMEM and leaks nothing, while
    tdh_pchol_noalloc makes no allocation at all (the injected failure stays pending)."""
    import torch
    n = 2000
    _, h, _, _ = tdh.symbols("leg2cheb", n)
    u = torch.zeros((32, n), dtype=torch.float64, device="cuda")
    piv = torch.zeros(32, dtype=torch.int64, device="cuda")
    K = ctypes.c_int64(-1)
    args = (ctypes.c_void_p(h.data_ptr()), n, 0, 1e-12, 32, ctypes.c_void_p(u.data_ptr()),
            ctypes.c_void_p(piv.data_ptr()), ctypes.byref(K), None)
    torch.cuda.synchronize()
    made0, live0, _ = tdh.alloc_stats()
    for k in (1, 2, 3):
        tdh.inject_alloc_failure(k)
        rc = tdh.lib().tdh_pchol(*args)
        tdh.inject_alloc_failure(0)
        if rc == 0:  # fewer allocations than k
            break
        assert rc == NOMEM, tdh.lib().tdh_last_error()
        assert tdh.alloc_stats()[1] == live0
    tdh.inject_alloc_failure(1)
    made = tdh.alloc_stats()[0]
    rc = tdh.lib().tdh_pchol_noalloc(*args)
    torch.cuda.synchronize()
    tdh.inject_alloc_failure(0)
    assert rc == 0, tdh.lib().tdh_last_error()
    assert tdh.alloc_stats()[0] == made


def test_tensor_core_wait_times_out_and_reports(tdh):
    """A split-bfloat16 execute whose tensor-core products are never issued (test hook): every
    CTA's bounded wait runs out after about a second, the kernel finishes, TIMEOUT is read
    back on the host, and the context stays usable (the next execute is correct)."""
    import time
    import torch
    import oracle
    import workloads
    n = 1000
    alpha = workloads.coefficients(n, 1, decay=1.0, seed=44)
    plan = tdh.Plan("leg2cheb", n, prec="bf16x3")
    x = torch.tensor(alpha, dtype=torch.float32, device="cuda")
    assert plan.status() == set()
    tdh.inject_tc_stall(True)
    try:
        t0 = time.perf_counter()
        plan.execute(x)
        torch.cuda.synchronize()
        waited = time.perf_counter() - t0
    finally:
        tdh.inject_tc_stall(False)
    assert plan.status() == {"TIMEOUT"}
    assert 0.5 <= waited <= 30.0, waited
    y = plan.execute(x)
    torch.cuda.synchronize()
    assert plan.status() == set()
    ref = oracle.matvec(oracle.LEG2CHEB, None, alpha)
    assert np.abs(y.double().cpu().numpy() - ref).max() / np.abs(alpha).sum() <= 1e-5
