"""The split-bfloat16 tensor-core execute (TDH_BF16X3) against the oracle (needs a GPU).

In these plans the radix-16 (radix-8) middle passes of every FFT within one cluster run as
DFT matrix products on the tensor cores (tcgen05), each operand split into bfloat16 hi and
lo parts and three products accumulated in float32; everything else is float32.  The stated
tolerance is max|beta - beta_ref| <= 1e-5 ||alpha||_1.  Covered: every compiled tensor-core
schedule (FFT lengths 2^8 ... 2^17, single CTAs and clusters of 2, 4, 8, forward and
transpose), both directions at the config-2 size, the config-3 ragged batch (4096 vectors,
one CUDA graph), an ultraspherical Case-2 step, and the float32 multi-pass fall-back beyond
one cluster.  No tensor-core wait may time out (tdh_plan_status).
"""
import numpy as np
import pytest

import oracle
import workloads

pytestmark = pytest.mark.gpu

TOL = 1e-5
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


def _rows(n, seed=0):
    if n <= 5000:
        return None
    rng = np.random.default_rng(seed)
    return np.unique(np.r_[np.arange(48), n - 1 - np.arange(48), rng.integers(0, n, 64)])


def _err(y, ref, alpha, rows):
    got = y if rows is None else y[:, rows]
    return (np.abs(got - ref).max(axis=-1) / np.abs(alpha).sum(axis=-1)).max()


# FFT lengths 2^8 ... 2^17 (parity packing: L = n for n a power of two), ragged tails
LENGTHS = [200, 300, 1000, 2000, 3000, 5000, 9000, 20000, 40000, 70000, 131072]


@pytest.mark.parametrize("n", LENGTHS)
def test_every_tensor_core_schedule(tdh, n):
    """Forward and transpose products on each tensor-core schedule of the plan's length."""
    import torch
    kind = "leg2cheb" if n % 2 == 0 else "cheb2leg"
    alpha = workloads.coefficients(n, 3, decay=0.5, seed=41)
    rows = _rows(n)
    ref = oracle.matvec(OKIND[kind], None, alpha, rows=rows)
    ref_t = oracle.matvec(OKIND[kind], None, alpha, rows=rows, transpose=True)
    plan = tdh.Plan(kind, n, prec="bf16x3")
    x = torch.tensor(alpha, dtype=torch.float32, device="cuda")
    count = plan.schedules()[0]["count"]
    compiled = tdh.compiled_schedules("bf16x3", plan.schedules()[0]["logL"])
    assert len(compiled) == count
    seen = set()
    for i in range(count):
        plan.set_schedule(i)
        s = plan.schedules()[0]
        seen.add((s["logLC"], s["C"], s["R"], s["NT"], s["MINB"], compiled[i]["multipass"]))
        y = plan.execute(x)
        g = plan.adjoint(x)
        torch.cuda.synchronize()
        e = _err(y.double().cpu().numpy(), ref, alpha, rows)
        et = _err(g.double().cpu().numpy(), ref_t, alpha, rows)
        assert e <= TOL and et <= TOL, (s, e, et)
    assert len(seen) == count
    assert plan.status() == set()


def test_every_compiled_tensor_core_schedule_is_reached(tdh):
    """The lengths above put a plan on every entry of the tensor-core schedule table."""
    want = set()
    for logL in range(8, 18):
        for s in tdh.compiled_schedules("bf16x3", logL):
            if not s["multipass"]:
                want.add((s["logLC"], s["C"], s["NT"], s["MINB"]))
    got = set()
    for n in LENGTHS:
        m = (n + 1) // 2
        logL = 8
        while (1 << logL) < 2 * m - 1:
            logL += 1
        for s in tdh.compiled_schedules("bf16x3", logL):
            if not s["multipass"]:
                got.add((s["logLC"], s["C"], s["NT"], s["MINB"]))
    assert want == got and len(want) == 18


@pytest.mark.parametrize("kind", ["leg2cheb", "cheb2leg"])
def test_config2_bf16x3_n2p16_b256(tdh, kind):
    """Config 2's size: n = 2^16, batch 256, alpha_k = z_k / sqrt(k+1); the first and last
    vectors on sampled rows, against the float32 path too."""
    import torch
    n, batch = 1 << 16, 256
    alpha = workloads.coefficients(n, batch, decay=0.5, seed=0)
    rows = _rows(n, seed=3)
    x = torch.tensor(alpha, dtype=torch.float32, device="cuda")
    plan = tdh.Plan(kind, n, prec="bf16x3")
    plan.autotune(batch)
    y = plan.execute(x)
    torch.cuda.synchronize()
    sel = [0, batch - 1]
    ref = oracle.matvec(OKIND[kind], None, alpha[sel], rows=rows)
    assert _err(y.double().cpu().numpy()[sel], ref, alpha[sel], rows) <= TOL
    y32 = tdh.Plan(kind, n, prec="fp32").execute(x)
    torch.cuda.synchronize()
    d = (y - y32).abs().amax(dim=1).double().cpu().numpy() / np.abs(alpha).sum(axis=1)
    assert d.max() <= TOL
    assert plan.status() == set()


def test_config3_ragged_bf16x3(tdh):
    """Config 3: 4096 Legendre -> Chebyshev vectors, degrees log-uniform in [64, 65536),
    alpha_k = z_k / (k+1), one ragged call and its CUDA-graph replay (identical)."""
    import torch
    deg = workloads.ragged_degrees(4096, 64, 65536, seed=0)
    lengths = deg + 1
    x, offs = workloads.ragged_coefficients(lengths, decay=1.0, seed=0)
    plan = tdh.Plan("leg2cheb", int(lengths.max()), prec="bf16x3", ragged=True)
    plan.autotune(len(lengths))
    xt = torch.tensor(x, dtype=torch.float32, device="cuda")
    ot = torch.tensor(offs, dtype=torch.int64, device="cuda")
    y = plan.execute_ragged(xt, ot)
    torch.cuda.synchronize()
    yn = y.double().cpu().numpy()
    rng = np.random.default_rng(6)
    worst = 0.0
    for i in np.unique(np.r_[np.argmax(lengths), np.argmin(lengths), rng.integers(0, 4096, 22)]):
        a, b = int(offs[i]), int(offs[i + 1])
        rows = _rows(b - a, seed=int(i))
        ref = oracle.matvec(oracle.LEG2CHEB, None, x[a:b], rows=rows)
        got = yn[a:b] if rows is None else yn[a:b][rows]
        worst = max(worst, np.abs(got - ref).max() / np.abs(x[a:b]).sum())
    assert worst <= TOL, worst
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
    assert plan.status() == set()


def test_ultraspherical_case2_bf16x3(tdh):
    import torch
    n = 9001
    params = (0.25, 1.0)
    alpha = workloads.coefficients(n, 2, decay=1.5, seed=42)
    plan = tdh.Plan("ultra2ultra", n, prec="bf16x3", params=params)
    y = plan.execute(torch.tensor(alpha, dtype=torch.float32, device="cuda"))
    torch.cuda.synchronize()
    ref = oracle.matvec(oracle.ULTRA, params, alpha)
    assert _err(y.double().cpu().numpy(), ref, alpha, None) <= TOL


def test_multipass_beyond_one_cluster_runs_float32(tdh):
    """n = 2^18: the FFT needs 16 slices, beyond one cluster; those kernels are float32."""
    import torch
    n = 1 << 18
    alpha = workloads.coefficients(n, 2, decay=1.0, seed=43)
    plan = tdh.Plan("leg2cheb", n, prec="bf16x3")
    s = plan.schedules()[0]
    assert s["C"] > 8
    y = plan.execute(torch.tensor(alpha, dtype=torch.float32, device="cuda"))
    torch.cuda.synchronize()
    rows = _rows(n)
    ref = oracle.matvec(oracle.LEG2CHEB, None, alpha, rows=rows)
    assert _err(y.double().cpu().numpy(), ref, alpha, rows) <= 5e-6
