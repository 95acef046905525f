"""Ragged batches (vectors of different lengths in one call) against the oracle at each
vector's own length: the n-prefix of an n_max plan converts the n-problem (needs a GPU)."""
import numpy as np
import pytest

import oracle
import workloads

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-12, "fp32": 5e-6}
OKIND = {"leg2cheb": oracle.LEG2CHEB, "cheb2leg": oracle.CHEB2LEG}


@pytest.fixture(scope="module")
def tdh():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1604_07486_gb300 as m
    from paper_1604_07486_gb300 import build
    build.build()
    return m


def _check_vectors(y, x, offs, kind, idx, prec, max_dense=20000):
    worst = 0.0
    for i in idx:
        a, b = int(offs[i]), int(offs[i + 1])
        if b == a:
            continue
        n = b - a
        rows = None if n <= max_dense else np.unique(np.r_[np.arange(48), n - 1 - np.arange(48),
                                                            np.random.default_rng(i).integers(0, n, 64)])
        ref = oracle.matvec(OKIND[kind], None, x[a:b], rows=rows)
        got = y[a:b] if rows is None else y[a:b][rows]
        worst = max(worst, np.abs(got - ref).max() / max(np.abs(x[a:b]).sum(), 1e-300))
    assert worst <= TOL[prec], worst
    return worst


@pytest.mark.parametrize("kind", ["leg2cheb", "cheb2leg"])
@pytest.mark.parametrize("prec,tol", [("fp32", None), ("fp64", None)])
def test_ragged_small(tdh, kind, prec, tol):
    """Lengths 0, 1, 2, ... up to 20000 (several FFT length classes, ragged tails)."""
    import torch
    if tol is None:
        tol = {("leg2cheb", "fp64"): 1e-15, ("cheb2leg", "fp64"): 1e-17,
               ("leg2cheb", "fp32"): 1e-7, ("cheb2leg", "fp32"): 1e-10}[(kind, prec)]
    lengths = np.r_[[0, 1, 2, 3, 5, 128, 129, 257, 1000], workloads.ragged_degrees(40, 16, 20000, seed=3) + 1]
    x, offs = workloads.ragged_coefficients(lengths, decay=1.0, seed=2)
    plan = tdh.Plan(kind, int(lengths.max()), prec=prec, tol=tol, ragged=True)
    xt = torch.tensor(x, dtype=plan.dtype, device="cuda")
    ot = torch.tensor(offs, dtype=torch.int64, device="cuda")
    y = plan.execute_ragged(xt, ot)
    torch.cuda.synchronize()
    _check_vectors(y.double().cpu().numpy(), x, offs, kind, range(len(lengths)), prec)


def test_config3_ragged_4096(tdh):
    """4096 Legendre -> Chebyshev vectors, degrees log-uniform in [64, 65536), alpha_k =
    z_k/(k+1), float32: 24 vectors (the longest, the shortest and random ones) against the
    oracle; the batch is also replayed from a captured CUDA graph with identical results."""
    import torch
    deg = workloads.ragged_degrees(4096, 64, 65536, seed=0)
    lengths = deg + 1
    x, offs = workloads.ragged_coefficients(lengths, decay=1.0, seed=0)
    plan = tdh.Plan("leg2cheb", int(lengths.max()), prec="fp32", tol=1e-7, ragged=True)
    xt = torch.tensor(x, dtype=torch.float32, device="cuda")
    ot = torch.tensor(offs, dtype=torch.int64, device="cuda")
    y = plan.execute_ragged(xt, ot)
    torch.cuda.synchronize()
    yn = y.double().cpu().numpy()
    rng = np.random.default_rng(5)
    idx = np.unique(np.r_[np.argmax(lengths), np.argmin(lengths), rng.integers(0, 4096, 22)])
    _check_vectors(yn, x, offs, "leg2cheb", idx, "fp32")
    # CUDA graph: capture once, replay
    out = torch.empty_like(xt)
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        plan.execute_ragged(xt, ot, out=out)
    torch.cuda.current_stream().wait_stream(s)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        plan.execute_ragged(xt, ot, out=out)
    out.zero_()
    g.replay()
    torch.cuda.synchronize()
    assert torch.equal(out, y)


def test_ragged_requires_flag(tdh):
    import torch
    plan = tdh.Plan("leg2cheb", 100, prec="fp32")
    x = torch.zeros(100, device="cuda")
    offs = torch.tensor([0, 100], dtype=torch.int64, device="cuda")
    with pytest.raises(tdh.TdhError) as e:
        plan.execute_ragged(x, offs)
    assert e.value.code == -1


def test_ragged_concurrent_threads(tdh):
    """Two host threads convert ragged batches with one plan on two streams at once: the
    plan's fork/join events are taken in turn, and each result equals the one-thread result."""
    import threading
    import torch
    lengths = workloads.ragged_degrees(300, 16, 20000, seed=8) + 1
    x, offs = workloads.ragged_coefficients(lengths, decay=1.0, seed=9)
    plan = tdh.Plan("leg2cheb", int(lengths.max()), prec="fp32", tol=1e-7, ragged=True)
    xt = torch.tensor(x, dtype=torch.float32, device="cuda")
    ot = torch.tensor(offs, dtype=torch.int64, device="cuda")
    want = plan.execute_ragged(xt, ot)
    torch.cuda.synchronize()
    outs, errs = [None, None], []

    def work(i):
        try:
            s = torch.cuda.Stream()
            with torch.cuda.stream(s):
                o = torch.empty_like(xt)
                for _ in range(20):
                    plan.execute_ragged(xt, ot, out=o, stream=s)
            s.synchronize()
            outs[i] = o
        except Exception as e:  # reported below
            errs.append(e)

    th = [threading.Thread(target=work, args=(i,)) for i in range(2)]
    for t in th:
        t.start()
    for t in th:
        t.join()
    assert not errs, errs
    for o in outs:
        assert torch.equal(o, want)


def test_ragged_device_checks(tdh):
    """Checks that need the device-resident offsets run on the device and are reported by
    tdh_plan_status: a vector longer than n_max is left unwritten (LENGTH); out overlapping
    in converts nothing (ALIAS); in == out is rejected on the host."""
    import torch
    n = 1000
    plan = tdh.Plan("leg2cheb", n, prec="fp32", ragged=True)
    assert plan.status() == set()
    x = torch.randn(3 * n, device="cuda")
    y = torch.full_like(x, 7.0)
    offs = torch.tensor([0, 500, 500 + n + 1, 2 * n + 501], dtype=torch.int64, device="cuda")
    plan.execute_ragged(x, offs, out=y)
    assert plan.status() == {"LENGTH"}
    assert torch.all(y[500:500 + n + 1] == 7.0)  # the over-long vector is left as it was
    assert plan.status() == set()                # cleared by the read
    buf = torch.zeros(4 * n, device="cuda")
    buf[: 2 * n] = torch.randn(2 * n, device="cuda")
    offs2 = torch.tensor([0, n, 2 * n], dtype=torch.int64, device="cuda")
    before = buf.clone()
    plan.execute_ragged(buf[: 2 * n], offs2, out=buf[n:3 * n])
    assert plan.status() == {"ALIAS"}
    assert torch.equal(buf, before)
    with pytest.raises(tdh.TdhError) as e:
        plan.execute_ragged(buf[: 2 * n], offs2, out=buf[: 2 * n])
    assert e.value.code == -7


@pytest.mark.parametrize("pinned", [True, False], ids=["pinned", "pageable"])
def test_ragged_host_buffers_equal_device(tdh, pinned):
    """tdh_plan_execute_ragged_host: config 3's batch (4096 vectors, ~39M coefficients, so the
    chunked pipeline with four chunks of whole vectors) from host memory gives the device
    ragged path's results bit for bit; so does a small batch (one chunk) with zero-length
    vectors and a nonzero first offset."""
    import torch
    deg = workloads.ragged_degrees(4096, 64, 65536, seed=0)
    lengths = deg + 1
    x, offs = workloads.ragged_coefficients(lengths, decay=1.0, seed=0)
    plan = tdh.Plan("leg2cheb", int(lengths.max()), prec="fp32", tol=1e-7, ragged=True)
    xt = torch.tensor(x, dtype=torch.float32, device="cuda")
    ot = torch.tensor(offs, dtype=torch.int64, device="cuda")
    ref = plan.execute_ragged(xt, ot).cpu()
    hx = torch.tensor(x, dtype=torch.float32)
    ho = torch.tensor(offs, dtype=torch.int64)
    if pinned:
        hx = hx.pin_memory()
    y = plan.execute_ragged(hx, ho)
    torch.cuda.synchronize()
    assert torch.equal(y, ref)
    assert plan.status() == set()
    # small batch: one chunk; vectors start at offset 3; two empty vectors
    lens = np.array([0, 100, 2000, 0, 513])
    offs2 = np.r_[3, 3 + np.cumsum(lens)].astype(np.int64)
    x2 = torch.randn(int(offs2[-1]) + 5, dtype=torch.float32)
    y2 = torch.full_like(x2, 7.0)
    plan.execute_ragged(x2, torch.tensor(offs2), out=y2)
    ref2 = torch.full_like(x2, 7.0).cuda()
    plan.execute_ragged(x2.cuda(), torch.tensor(offs2, device="cuda"), out=ref2)
    torch.cuda.synchronize()
    assert torch.equal(y2, ref2.cpu())
    assert torch.all(y2[:3] == 7.0) and torch.all(y2[int(offs2[-1]):] == 7.0)


def test_ragged_host_argument_checks(tdh):
    """Host offsets are checked before anything runs: decreasing offsets, a negative first
    offset and a vector longer than n_max are INVALID_ARG; overlapping in and out are ALIAS;
    a scratch allocation failure is NOMEM and leaves nothing held."""
    import torch
    n = 1000
    plan = tdh.Plan("leg2cheb", n, prec="fp32", ragged=True)
    x = torch.randn(3 * n, dtype=torch.float32)
    y = torch.zeros_like(x)
    for bad in ([0, 500, 400], [-1, 500, 900], [0, 500, 500 + n + 1]):
        with pytest.raises(tdh.TdhError) as e:
            plan.execute_ragged(x, torch.tensor(bad, dtype=torch.int64), out=y)
        assert e.value.code == -1, bad
    assert torch.all(y == 0)
    buf = torch.randn(4 * n, dtype=torch.float32)
    with pytest.raises(tdh.TdhError) as e:
        plan.execute_ragged(buf[: 2 * n], torch.tensor([0, n, 2 * n]), out=buf[n:3 * n])
    assert e.value.code == -7
    _, live0, scr0 = tdh.alloc_stats()
    tdh.inject_alloc_failure(1)
    try:
        with pytest.raises(tdh.TdhError) as e:
            plan.execute_ragged(x, torch.tensor([0, n, 2 * n, 3 * n]), out=y)
    finally:
        tdh.inject_alloc_failure(0)
    assert e.value.code == -3
    torch.cuda.synchronize()
    assert tdh.alloc_stats()[1:] == (live0, scr0)
    plan.execute_ragged(x, torch.tensor([0, n, 2 * n, 3 * n]), out=y)
    torch.cuda.synchronize()
    ref = plan.execute_ragged(x.cuda(), torch.tensor([0, n, 2 * n, 3 * n], device="cuda")).cpu()
    assert torch.equal(y, ref)


@pytest.mark.parametrize("prec", ["fp64", "bf16x3"])
def test_ragged_host_buffers_other_precisions(tdh, prec):
    """The host-buffer ragged path in float64 and with split-bfloat16 passes: 1000 vectors
    (~9M coefficients, above 24 MB in either precision, so chunked) equal the device path bit
    for bit."""
    import torch
    lengths = workloads.ragged_degrees(1000, 64, 65536, seed=7) + 1
    x, offs = workloads.ragged_coefficients(lengths, decay=1.0, seed=7)
    plan = tdh.Plan("leg2cheb", int(lengths.max()), prec=prec, ragged=True)
    dt = torch.float64 if prec == "fp64" else torch.float32
    ref = plan.execute_ragged(torch.tensor(x, dtype=dt, device="cuda"),
                              torch.tensor(offs, dtype=torch.int64, device="cuda")).cpu()
    y = plan.execute_ragged(torch.tensor(x, dtype=dt).pin_memory(),
                            torch.tensor(offs, dtype=torch.int64))
    torch.cuda.synchronize()
    assert torch.equal(y, ref)
    assert plan.status() == set()
