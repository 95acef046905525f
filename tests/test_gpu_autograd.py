"""Differentiable Legendre -> Chebyshev (n = 8192, batch 1024, float32): the backward adjoint
kernel against the dense float64 A^T of the oracle and against central finite differences
(h = 1e-3, float64 plan)."""
import numpy as np
import pytest

import oracle
import workloads

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


def _loss(beta, torch):
    k = torch.arange(beta.shape[-1], device=beta.device, dtype=beta.dtype)
    return ((k + 1.0) ** 2 * beta * beta).sum()


def test_config5_gradient_vs_dense_adjoint(tdh):
    """loss = sum_k (k+1)^2 beta_k^2; grad = A^T (2 (k+1)^2 beta).  The float32 gradient of the
    whole batch equals the oracle's dense A^T applied to the same cotangent (sampled vectors)."""
    import torch
    from paper_1604_07486_gb300.autograd import convert
    n, batch = 8192, 1024
    plan = tdh.Plan("leg2cheb", n, prec="fp32", tol=1e-7)
    alpha = workloads.coefficients(n, batch, decay=1.0, seed=0)
    x = torch.tensor(alpha, dtype=torch.float32, device="cuda", requires_grad=True)
    beta = convert(x, plan)
    loss = _loss(beta, torch)
    loss.backward()
    g = x.grad.double().cpu().numpy()
    cot = (2.0 * (np.arange(n) + 1.0) ** 2 * beta.detach().double().cpu().numpy())
    vecs = np.array([0, 511, 1023])
    ref = oracle.matvec(oracle.LEG2CHEB, None, cot[vecs], transpose=True)
    err = (np.abs(g[vecs] - ref).max(axis=1) / np.abs(cot[vecs]).sum(axis=1)).max()
    assert err <= 5e-6, err


def test_gradient_vs_central_differences(tdh):
    """Central differences of the loss in float64 (h = 1e-3) along random directions agree with
    <grad, direction> from the adjoint kernel."""
    import torch
    from paper_1604_07486_gb300.autograd import convert
    n, batch = 8192, 4
    plan = tdh.Plan("leg2cheb", n, prec="fp64", tol=1e-15)
    alpha = workloads.coefficients(n, batch, decay=1.0, seed=1)
    x = torch.tensor(alpha, dtype=torch.float64, device="cuda", requires_grad=True)
    loss = _loss(convert(x, plan), torch)
    loss.backward()
    g = x.grad.detach()
    rng = np.random.default_rng(9)
    h = 1e-3
    for _ in range(3):
        d = torch.tensor(rng.standard_normal((batch, n)), dtype=torch.float64, device="cuda")
        with torch.no_grad():
            lp = _loss(plan.execute((x + h * d).contiguous()), torch)
            lm = _loss(plan.execute((x - h * d).contiguous()), torch)
        fd = float((lp - lm) / (2 * h))
        an = float((g * d).sum())
        assert abs(fd - an) <= 1e-7 * abs(an) + 1e-9, (fd, an)


def test_gradcheck_small(tdh):
    """torch.autograd.gradcheck on a small float64 Chebyshev -> Legendre plan."""
    import torch
    from paper_1604_07486_gb300.autograd import convert
    plan = tdh.Plan("cheb2leg", 40, prec="fp64", tol=1e-17)
    x = torch.tensor(workloads.coefficients(40, 2, seed=2), dtype=torch.float64, device="cuda",
                     requires_grad=True)
    assert torch.autograd.gradcheck(lambda a: convert(a, plan), (x,), eps=1e-6, atol=1e-8)


@pytest.mark.parametrize("kind,params", [("jac2jac", (0.5, 0.25, 2.5, 0.25)),
                                         ("jac2jac", (1.75, 0.5, -0.5, 0.25)),
                                         ("ultra2ultra", (2.25, 0.75)),
                                         ("jac2cheb", (0.25, -0.3)),
                                         ("lag2lag", (0.5, -0.25))],
                         ids=["jacobi_whole_steps", "jacobi_mixed_chain", "ultra_downward",
                              "jac2cheb", "laguerre"])
def test_gradcheck_chains(tdh, kind, params):
    """gradcheck through chains with sparse factors, back-substitution, reflections and the
    Chebyshev normalisation (float64, small n: the adjoint of every step kind)."""
    import torch
    from paper_1604_07486_gb300.autograd import convert
    plan = tdh.Plan(kind, 37, prec="fp64", tol=1e-16, params=params)
    x = torch.tensor(workloads.coefficients(37, 2, seed=3), dtype=torch.float64, device="cuda",
                     requires_grad=True)
    assert torch.autograd.gradcheck(lambda a: convert(a, plan), (x,), eps=1e-6, atol=1e-7)
