"""Every compiled execute schedule (local FFT length, cluster size, threads, CTAs per SM, and
for multi-pass lengths the cross stage with or without bulk tensor copies) and the autotuner
against the oracle (needs a GPU).

A schedule changes only the order of the FFT's floating-point operations, so each one must
meet the same tolerance (max |beta - beta_ref| / ||alpha||_1: float64 1e-12, float32 5e-6).
The lengths below put at least one plan on every schedule of the table: FFT lengths 2^8 ...
2^18, single CTAs, clusters of 2/4/8 (radix 16 and radix 32) and the multi-pass kernels on
full and half slices.
"""
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


def _rows(n, seed=0):
    if n <= 5000:
        return None
    rng = np.random.default_rng(seed)
    return np.unique(np.r_[np.arange(48), n - 1 - np.arange(48), rng.integers(0, n, 64)])


def _err(y, ref, alpha, rows):
    got = y if rows is None else y[:, rows]
    return (np.abs(got - ref).max(axis=-1) / np.abs(alpha).sum(axis=-1)).max()


CASES = [("leg2cheb", n, "fp32") for n in (200, 300, 1000, 2000, 3000, 5000, 9000, 20000, 70000)]
CASES += [("cheb2leg", 40000, "fp32"), ("leg2cheb", 1 << 18, "fp32")]
CASES += [("leg2cheb", n, "fp64") for n in (200, 300, 1000, 2000, 3000, 5000, 9000, 20000, 40000)]


@pytest.mark.parametrize("kind,n,prec", CASES)
def test_every_schedule(tdh, kind, n, prec):
    """Forward and transpose products on each schedule of the plan's FFT length."""
    import torch
    tol = {"fp32": 1e-7, "fp64": 1e-15}[prec] if kind == "leg2cheb" else 1e-10
    batch = 3
    alpha = workloads.coefficients(n, batch, decay=0.5, seed=11)
    rows = _rows(n)
    ref = oracle.matvec(OKIND[kind], None, alpha, rows=rows)
    ref_t = oracle.matvec(OKIND[kind], None, alpha, rows=rows, transpose=True)
    plan = tdh.Plan(kind, n, prec=prec, tol=tol)
    x = torch.tensor(alpha, dtype=plan.dtype, device="cuda")
    count = plan.schedules()[0]["count"]
    assert count >= 2, plan.schedules()
    compiled = tdh.compiled_schedules(prec, plan.schedules()[0]["logL"])
    assert len(compiled) == count
    seen = set()
    for i in range(count):
        plan.set_schedule(i)
        s = plan.schedules()[0]
        assert s["index"] == i and s["count"] == count, s
        assert (1 << s["logLC"]) * s["C"] == 1 << s["logL"], s
        c = compiled[i]
        assert (c["logLC"], c["C"], c["R"], c["NT"], c["MINB"]) == \
            (s["logLC"], s["C"], s["R"], s["NT"], s["MINB"])
        seen.add((s["logLC"], s["C"], s["R"], s["NT"], s["MINB"], c["multipass"]))
        y = plan.execute(x)
        g = plan.adjoint(x)
        torch.cuda.synchronize()
        e = _err(y.double().cpu().numpy(), ref, alpha, rows)
        et = _err(g.double().cpu().numpy(), ref_t, alpha, rows)
        assert e <= TOL[prec] and et <= TOL[prec], (s, e, et)
    assert len(seen) == count
    assert plan.status() == set()  # no bounded wait ran out, no copy was skipped
    # indices past the end take the last schedule
    plan.set_schedule(count + 5)
    assert plan.schedules()[0]["index"] == count - 1


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_ragged_every_schedule(tdh, prec):
    """A ragged batch (FFT length classes 2^8 ... 2^15) on each schedule index."""
    import torch
    lengths = np.r_[[0, 1, 2, 129, 257, 700, 1500, 3000, 6000, 9000, 15000, 20000],
                    workloads.ragged_degrees(20, 16, 20000, seed=5) + 1]
    x, offs = workloads.ragged_coefficients(lengths, decay=1.0, seed=4)
    plan = tdh.Plan("leg2cheb", int(lengths.max()), prec=prec,
                    tol={"fp32": 1e-7, "fp64": 1e-15}[prec], ragged=True)
    xt = torch.tensor(x, dtype=plan.dtype, device="cuda")
    ot = torch.tensor(offs, dtype=torch.int64, device="cuda")
    refs = {}
    for v in range(len(lengths)):
        a, b = int(offs[v]), int(offs[v + 1])
        if b > a:
            rows = _rows(b - a, seed=v)
            refs[v] = (rows, oracle.matvec(oracle.LEG2CHEB, None, x[a:b], rows=rows))
    sched = plan.schedules()
    assert len(sched) == 1 + (15 - 8 + 1), sched  # dense configuration + classes 2^8..2^15
    top = max(s["count"] for s in sched)
    for i in range(top):
        plan.set_schedule(i)
        for s in plan.schedules()[1:]:
            assert s["C"] <= 8 and s["index"] == min(i, s["count"] - 1), s
        y = plan.execute_ragged(xt, ot).double().cpu().numpy()
        worst = 0.0
        for v, (rows, ref) in refs.items():
            a, b = int(offs[v]), int(offs[v + 1])
            got = y[a:b] if rows is None else y[a:b][rows]
            worst = max(worst, np.abs(got - ref).max() / np.abs(x[a:b]).sum())
        assert worst <= TOL[prec], (i, worst)


def test_autotune_dense_and_ragged(tdh):
    """The autotuner keeps one compiled schedule per configuration and the results still
    match the oracle; tuning is repeatable in what it reports about the schedule space."""
    import torch
    n, batch = 20000, 8
    alpha = workloads.coefficients(n, batch, decay=0.5, seed=12)
    rows = _rows(n)
    ref = oracle.matvec(oracle.LEG2CHEB, None, alpha, rows=rows)
    plan = tdh.Plan("leg2cheb", n, prec="fp32", tol=1e-7, ragged=True)
    before = plan.schedules()
    after = plan.autotune(batch)
    assert len(after) == len(before)
    for b, a in zip(before, after):
        assert a["logL"] == b["logL"] and a["count"] == b["count"]
        assert 0 <= a["index"] < a["count"]
    x = torch.tensor(alpha, dtype=torch.float32, device="cuda")
    y = plan.execute(x).double().cpu().numpy()
    assert _err(y, ref, alpha, rows) <= TOL["fp32"]
    offs = torch.arange(0, (batch + 1) * n, n, dtype=torch.int64, device="cuda")
    yr = plan.execute_ragged(x.reshape(-1), offs).double().cpu().numpy().reshape(batch, n)
    assert _err(yr, ref, alpha, rows) <= TOL["fp32"]


def test_autotune_chain(tdh):
    """A Jacobi chain (two T o H steps and rank-pair packing) after tuning each step."""
    import torch
    n, batch = 4096, 2
    a, b, g, d = 0.1, -0.3, 0.0, 0.0
    alpha = workloads.coefficients(n, batch, decay=1.5, seed=13)
    ref = np.stack([oracle.jac2jac(v, a, b, g, d) for v in alpha])
    plan = tdh.Plan("jac2jac", n, prec="fp64", tol=1e-15, params=(a, b, g, d))
    sched = plan.autotune(batch)
    assert len(sched) == 2, sched
    y = plan.execute(torch.tensor(alpha, dtype=torch.float64, device="cuda"))
    assert _err(y.double().cpu().numpy(), ref, alpha, None) <= TOL["fp64"]


def test_schedule_errors(tdh):
    plan = tdh.Plan("leg2cheb", 1000, prec="fp32")
    with pytest.raises(tdh.TdhError):
        plan.set_schedule(-1)
    with pytest.raises(tdh.TdhError):
        plan.autotune(0)
    import ctypes
    info = (ctypes.c_int * 8)()
    assert tdh.lib().tdh_plan_schedule_info(plan._h, 1, info) == -1


def test_plans_without_fft_steps(tdh):
    """A conversion made only of banded factors (ultraspherical 0.25 -> 1.25, Case 1) has no
    execute configuration: the schedule calls have nothing to do and succeed."""
    import torch
    n = 4096
    plan = tdh.Plan("ultra2ultra", n, prec="fp32", tol=1e-13, params=(0.25, 1.25))
    assert plan.schedules() == []
    plan.set_schedule(3)
    assert plan.autotune(4) == []
    alpha = workloads.coefficients(n, 2, decay=1.0, seed=14)
    ref = oracle.matvec(oracle.ULTRA, (0.25, 1.25), alpha)
    y = plan.execute(torch.tensor(alpha, dtype=torch.float32, device="cuda"))
    assert _err(y.double().cpu().numpy(), ref, alpha, None) <= TOL["fp32"]
