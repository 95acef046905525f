"""CUDA path against the CPU oracle, element by element (needs a GPU).

Tolerances (max |beta - beta_ref| / ||alpha||_1): float64 1e-12, float32 5e-6.  Inputs are the
seeded workloads of workloads.py.  Each step of the path is checked on its own through the
C ABI (symbols a1, pivoted Cholesky a2) and end to end (a3-a7).
"""
import numpy as np
import pytest

import oracle
import workloads

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-12, "fp32": 5e-6}
OKIND = {"leg2cheb": oracle.LEG2CHEB, "cheb2leg": oracle.CHEB2LEG, "ultra2ultra": oracle.ULTRA}


@pytest.fixture(scope="module")
def tdh():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1604_07486_gb300 as m
    from paper_1604_07486_gb300 import build
    build.build()
    return m


def _torch():
    import torch
    return torch


def _rel_err(y, ref, alpha):
    return (np.abs(y - ref).max(axis=-1) / np.abs(alpha).sum(axis=-1)).max()


def _run(tdh, kind, n, batch, prec, tol, decay=1.0, params=(), seed=0):
    torch = _torch()
    alpha = workloads.coefficients(n, batch, decay=decay, seed=seed)
    plan = tdh.Plan(kind, n, prec=prec, tol=tol, params=params)
    x = torch.tensor(alpha, dtype=plan.dtype, device="cuda")
    y = plan.execute(x)
    torch.cuda.synchronize()
    return plan, alpha, y.double().cpu().numpy()


# ------------------------------------------------------------------------------- a1

@pytest.mark.parametrize("kind,params", [("leg2cheb", ()), ("cheb2leg", ()),
                                         ("ultra2ultra", (0.75, 1.25)),
                                         ("jac2jac", (0.1, -0.3, 0.0))])
@pytest.mark.parametrize("n", [37, 4096, 1 << 20])
def test_symbols(tdh, kind, params, n):
    """Gamma-ratio symbols on the GPU (asymptotic series) vs the oracle's double-double
    recurrences: a few ulp relative, including arguments near 2^20 where log-gamma
    differences would lose five digits."""
    okind = {"leg2cheb": oracle.LEG2CHEB, "cheb2leg": oracle.CHEB2LEG,
             "ultra2ultra": oracle.ULTRA, "jac2jac": oracle.JAC}[kind]
    got = [a.cpu().numpy() for a in tdh.symbols(kind, n, params)]
    ref = oracle.split(okind, params, n)
    for name, g, r in zip(("t", "h", "d1", "d2"), got, ref):
        scale = np.maximum(np.abs(r), 1e-300)
        rel = (np.abs(g - r) / scale).max()
        assert rel < 2e-14, (name, rel)
        assert np.array_equal(g == 0, r == 0), name


# ------------------------------------------------------------------------------- a2

@pytest.mark.parametrize("kind,j0", [("leg2cheb", 0), ("cheb2leg", 1)])
@pytest.mark.parametrize("n,tol", [(301, 1e-15), (5000, 1e-10), (65536, 1e-15)])
def test_pchol(tdh, kind, j0, n, tol):
    """GPU pivoted Cholesky on the oracle's Hankel generator vs the oracle's Fig. 2 algorithm:
    same pivots, same rank (up to the last step near the threshold), same factors."""
    torch = _torch()
    okind = OKIND[kind]
    _, h, _, _ = oracle.split(okind, None, n)
    u, piv = tdh.pchol(torch.tensor(h, device="cuda"), n, j0, tol)
    u, piv = u.cpu().numpy(), piv.cpu().numpy()
    ur, pr = oracle.hankel_factors(okind, None, n, tol)
    assert abs(len(piv) - len(pr)) <= 1 and min(len(piv), len(pr)) >= 10
    # steps whose pivot is far above the rounding level are deterministic: same pivot and
    # same column; later ones may legitimately differ in rounding
    a = np.array([ur[r, pr[r]] ** 2 for r in range(len(pr))])
    K = int(np.sum(a > 1e-8 * a[0]))
    assert np.array_equal(piv[:K], pr[:K])
    assert np.abs(u[:K] - ur[:K]).max() < 1e-9 * np.abs(ur).max()
    # the approximation itself on a sampled block
    rng = np.random.default_rng(0)
    rows = np.sort(rng.choice(np.arange(j0, n), size=min(200, n - j0), replace=False))
    Hb = h[rows[:, None] + rows[None, :]]
    approx = u[:, rows].T @ u[:, rows]
    assert np.abs(Hb - approx).max() <= 4 * tol * h[2 * j0]


# ---------------------------------------------------------------------------- a3-a6

@pytest.mark.parametrize("kind", ["leg2cheb", "cheb2leg"])
@pytest.mark.parametrize("prec,tol", [("fp64", None), ("fp32", None)])
@pytest.mark.parametrize("n", [1, 2, 3, 7, 100, 256, 257, 1000, 1024, 4097, 8192, 16385, 30000])
def test_execute_small(tdh, kind, prec, tol, n):
    """Dense oracle on every row, several tiles and ragged tails, both directions."""
    if tol is None:
        tol = {("leg2cheb", "fp64"): 1e-15, ("cheb2leg", "fp64"): 1e-17,
               ("leg2cheb", "fp32"): 1e-7, ("cheb2leg", "fp32"): 1e-10}[(kind, prec)]
    batch = 3
    plan, alpha, y = _run(tdh, kind, n, batch, prec, tol, decay=0.5)
    ref = oracle.matvec(OKIND[kind], None, alpha)
    err = _rel_err(y, ref, alpha)
    assert err <= TOL[prec], (err, plan.K)


def test_config1_leg2cheb_n1024_fp64(tdh):
    """Legendre -> Chebyshev, n = 1024, one vector, float64, alpha_k = z_k/(k+1), tol 1e-15."""
    plan, alpha, y = _run(tdh, "leg2cheb", 1024, 1, "fp64", 1e-15, decay=1.0)
    ref = oracle.matvec(oracle.LEG2CHEB, None, alpha)
    assert _rel_err(y, ref, alpha) <= 1e-12
    assert 20 <= plan.K <= 40


@pytest.mark.parametrize("kind,prec,tol", [("leg2cheb", "fp32", 1e-7), ("leg2cheb", "fp64", 1e-15),
                                           ("cheb2leg", "fp32", 1e-10), ("cheb2leg", "fp64", 1e-17)])
def test_config2_n65536_single_vector_dense(tdh, kind, prec, tol):
    """n = 2^16, one vector, alpha_k = z_k/(k+1)^0.5: every row against the dense oracle."""
    plan, alpha, y = _run(tdh, kind, 1 << 16, 1, prec, tol, decay=0.5)
    ref = oracle.matvec(OKIND[kind], None, alpha)
    assert _rel_err(y, ref, alpha) <= TOL[prec]


@pytest.mark.parametrize("kind,prec,tol", [("leg2cheb", "fp32", 1e-7), ("cheb2leg", "fp32", 1e-10),
                                           ("leg2cheb", "fp64", 1e-15)])
def test_config2_n65536_batch256_sampled(tdh, kind, prec, tol):
    """The bench's launch: batch 256 of n = 2^16.  Sampled rows (first, last, random) of
    eight vectors spread over the batch against the oracle, row by row."""
    n, batch = 1 << 16, 256
    plan, alpha, y = _run(tdh, kind, n, batch, prec, tol, decay=0.5)
    rng = np.random.default_rng(1)
    rows = np.unique(np.concatenate([np.arange(64), n - 1 - np.arange(64),
                                     rng.integers(0, n, 128)]))
    vecs = np.array([0, 37, 100, 128, 200, 254, 255, 17])
    ref = oracle.matvec(OKIND[kind], None, alpha[vecs], rows=rows)
    err = (np.abs(y[vecs][:, rows] - ref).max(axis=1) / np.abs(alpha[vecs]).sum(axis=1)).max()
    assert err <= TOL[prec]
    assert np.all(np.isfinite(y))


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-15), ("fp32", 1e-7)])
def test_ultraspherical_case2(tdh, prec, tol):
    """C^(3/4) -> C^(5/4) (Sec. 5.2 Case 2) against the dense oracle."""
    n = 5000
    plan, alpha, y = _run(tdh, "ultra2ultra", n, 2, prec, tol, decay=1.0, params=(0.75, 1.25))
    ref = oracle.matvec(oracle.ULTRA, (0.75, 1.25), alpha)
    assert _rel_err(y, ref, alpha) <= TOL[prec]


# ------------------------------------------------------------------------------- a7

@pytest.mark.parametrize("kind", ["leg2cheb", "cheb2leg"])
@pytest.mark.parametrize("prec,tol", [("fp64", None), ("fp32", None)])
@pytest.mark.parametrize("n", [5, 1000, 8192, 40000])
def test_adjoint(tdh, kind, prec, tol, n):
    """A^T g against the oracle's dense transpose, and <A a, g> = <a, A^T g>."""
    torch = _torch()
    if tol is None:
        tol = {("leg2cheb", "fp64"): 1e-15, ("cheb2leg", "fp64"): 1e-17,
               ("leg2cheb", "fp32"): 1e-7, ("cheb2leg", "fp32"): 1e-10}[(kind, prec)]
    plan = tdh.Plan(kind, n, prec=prec, tol=tol)
    g = workloads.cotangent(n, 2, seed=3)
    a = workloads.coefficients(n, 2, decay=1.0, seed=4)
    gt = torch.tensor(g, dtype=plan.dtype, device="cuda")
    at = torch.tensor(a, dtype=plan.dtype, device="cuda")
    atg = plan.adjoint(gt).double().cpu().numpy()
    aa = plan.execute(at).double().cpu().numpy()
    rows = np.arange(n) if n <= 8192 else np.unique(np.r_[np.arange(100), n - 1 - np.arange(100),
                                                         np.random.default_rng(2).integers(0, n, 200)])
    ref = oracle.matvec(OKIND[kind], None, g, rows=rows, transpose=True)
    err = (np.abs(atg[:, rows] - ref).max(axis=1) / np.abs(g).sum(axis=1)).max()
    assert err <= TOL[prec], err
    lhs = (aa * g).sum(axis=1)
    rhs = (a * atg).sum(axis=1)
    scale = np.abs(aa).sum(axis=1) * np.abs(g).max(axis=1) + np.abs(a).sum(axis=1) * np.abs(atg).max(axis=1)
    assert np.all(np.abs(lhs - rhs) <= 10 * TOL[prec] * scale)


# ------------------------------------------------------------------------------- errors

def test_error_paths(tdh):
    torch = _torch()
    plan = tdh.Plan("leg2cheb", 100, prec="fp32")
    x = torch.zeros(2, 100, device="cuda")
    assert tdh.lib().tdh_plan_execute(plan._h, None, None, 1, None) == -1
    buf = torch.zeros(1000, device="cuda")
    import ctypes
    rc = tdh.lib().tdh_plan_execute(plan._h, ctypes.c_void_p(buf.data_ptr() + 4),
                                    ctypes.c_void_p(buf.data_ptr() + 512), 1, None)
    assert rc == -4
    rc = tdh.lib().tdh_plan_execute(plan._h, ctypes.c_void_p(buf.data_ptr()),
                                    ctypes.c_void_p(buf.data_ptr() + 256), 1, None)
    assert rc == -7
    assert tdh.lib().tdh_plan_execute(plan._h, ctypes.c_void_p(buf.data_ptr()),
                                      ctypes.c_void_p(buf.data_ptr() + 1024), 0, None) == 0
    with pytest.raises(tdh.TdhError) as e:
        tdh.Plan("jac2jac", 100, params=(-1.0, 0.0, 1.6, 0.0))  # a <= -1
    assert e.value.code == -1
    with pytest.raises(tdh.TdhError):
        tdh.Plan("ultra2ultra", 100, params=(-1.0, 0.5))
    with pytest.raises(tdh.TdhError) as e:  # ragged batches need one T o H step
        tdh.Plan("ultra2ultra", 100, params=(0.25, 1.25), ragged=True)
    assert e.value.code == -2
    y = plan.execute(x)
    torch.cuda.synchronize()
    assert torch.all(y == 0)


# ------------------------------------------------------------------------------- Jacobi

JAC_CASES = [
    ((0.1, -0.3, 0.0, -0.3), "one Case-2 step (b = d)"),
    ((0.1, -0.3, 0.0, 0.0), "reflection chain: (0.1,-0.3) -> (0.1,0) -> (0,0)"),
    ((0.0, 2 ** 0.5 / 2, -0.25, 2 ** 0.5 / 2), "the paper's Fig. 6 workload"),
    ((-0.4, -0.5, 0.25, -0.5), "near the Chebyshev weight"),
    ((-0.5, -0.5, 0.25, -0.5), "Case 3 from the Chebyshev weight"),
    ((-0.6, -0.7, -0.2, -0.7), "Case 3"),
    ((-0.5, -0.5, 0.0, 0.0), "chain with a Case-3 reflection step"),
]


@pytest.mark.parametrize("params,desc", JAC_CASES, ids=[c[1] for c in JAC_CASES])
@pytest.mark.parametrize("prec,tol,n", [("fp64", 1e-15, 3001), ("fp32", 1e-13, 3001),
                                        ("fp32", 1e-13, 40000)])
def test_jacobi(tdh, params, desc, prec, tol, n):
    """Jacobi conversion (Sec. 5.3): no parity structure, so rank terms are packed in pairs;
    b != d runs the reflection chain.  Dense oracle chain (pinned by exact rationals)."""
    torch = _torch()
    a, b, g, d = params
    alpha = workloads.coefficients(n, 2, decay=1.5, seed=5)
    plan = tdh.Plan("jac2jac", n, prec=prec, tol=tol, params=params)
    y = plan.execute(torch.tensor(alpha, dtype=plan.dtype, device="cuda"))
    torch.cuda.synchronize()
    y = y.double().cpu().numpy()
    rows = None if n <= 4096 else np.unique(np.r_[np.arange(64), n - 1 - np.arange(64),
                                                  np.random.default_rng(4).integers(0, n, 128)])
    if b == d:
        ref = oracle.matvec(oracle.JAC, (a, b, g), alpha, rows=rows)
    else:
        ref = np.stack([oracle.jac2jac(v, a, b, g, d, rows=rows) for v in alpha])
    yy = y if rows is None else y[:, rows]
    err = (np.abs(yy - ref).max(axis=1) / np.abs(alpha).sum(axis=1)).max()
    assert err <= TOL[prec], (err, plan.K)


def test_jacobi_adjoint(tdh):
    """The chain's adjoint runs the steps in reverse: <A a, g> = <a, A^T g>."""
    torch = _torch()
    n = 2000
    plan = tdh.Plan("jac2jac", n, prec="fp64", tol=1e-15, params=(0.1, -0.3, 0.0, 0.0))
    a = torch.tensor(workloads.coefficients(n, 1, decay=1.0, seed=6), dtype=torch.float64, device="cuda")
    g = torch.tensor(workloads.cotangent(n, 1, seed=7), dtype=torch.float64, device="cuda")
    lhs = float((plan.execute(a) * g).sum())
    rhs = float((a * plan.adjoint(g)).sum())
    assert abs(lhs - rhs) <= 1e-11 * (abs(lhs) + 1.0)


# ------------------------------------------------------------------ ultraspherical Case 1/3

@pytest.mark.parametrize("params", [(0.25, 1.25), (0.25, 2.25), (0.25, 1.75), (0.6, 3.1)],
                         ids=["case1", "case1_two_factors", "case3", "case3_two_steps"])
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_ultraspherical_case1_case3(tdh, params, prec):
    """Sec. 5.2 Case 1 (sparse factors of Eq. (12)) and Case 3 (whole steps,
    then Case 2) against the dense oracle (Eq. (13) covers every case)."""
    n = 4099
    tol = 1e-15 if prec == "fp64" else 1e-8
    plan, alpha, y = _run(tdh, "ultra2ultra", n, 3, prec, tol, decay=1.5, params=params)
    ref = oracle.matvec(oracle.ULTRA, params, alpha)
    assert _rel_err(y, ref, alpha) <= TOL[prec]


def test_ultraspherical_case1_adjoint(tdh):
    torch = _torch()
    n = 3000
    plan = tdh.Plan("ultra2ultra", n, prec="fp64", params=(0.25, 2.25))
    g = workloads.cotangent(n, 2, seed=3)
    atg = plan.adjoint(torch.tensor(g, device="cuda")).cpu().numpy()
    ref = oracle.matvec(oracle.ULTRA, (0.25, 2.25), g, transpose=True)
    assert _rel_err(atg, ref, g) <= 1e-12


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_config4_ultraspherical_n2p20_b16(tdh, prec):
    """C^(0.25) -> C^(1.25) at n = 2^20, batch 16, alpha_k = z_k (k+1)^-1.5: sampled rows of
    every vector against the oracle (Case 1: one sparse factor)."""
    n, batch = 1 << 20, 16
    plan, alpha, y = _run(tdh, "ultra2ultra", n, batch, prec, 1e-13, decay=1.5, params=(0.25, 1.25))
    rows = np.unique(np.r_[np.arange(64), n - 1 - np.arange(64),
                           np.random.default_rng(8).integers(0, n, 256)])
    ref = oracle.matvec(oracle.ULTRA, (0.25, 1.25), alpha, rows=rows)
    err = (np.abs(y[:, rows] - ref).max(axis=1) / np.abs(alpha).sum(axis=1)).max()
    assert err <= TOL[prec]


# ---------------------------------------------------------------- multi-pass (large L)

def _rows(n, seed=4, k=64):
    return np.unique(np.r_[np.arange(k), n - 1 - np.arange(k),
                           np.random.default_rng(seed).integers(0, n, k)])


@pytest.mark.parametrize("kind,prec,tol,n", [("leg2cheb", "fp64", 1e-15, 70001),
                                             ("cheb2leg", "fp64", 1e-17, 70001),
                                             ("leg2cheb", "fp32", 1e-7, 200001),
                                             ("cheb2leg", "fp32", 1e-10, 200001)])
def test_multipass_parity(tdh, kind, prec, tol, n):
    """FFT lengths beyond one cluster (exchange through global memory): sampled rows against
    the oracle, and the adjoint identity."""
    torch = _torch()
    plan, alpha, y = _run(tdh, kind, n, 2, prec, tol, decay=0.5)
    rows = _rows(n)
    ref = oracle.matvec(OKIND[kind], None, alpha, rows=rows)
    err = (np.abs(y[:, rows] - ref).max(axis=1) / np.abs(alpha).sum(axis=1)).max()
    assert err <= TOL[prec], err
    g = workloads.cotangent(n, 2, seed=3)
    atg = plan.adjoint(torch.tensor(g, dtype=plan.dtype, device="cuda")).double().cpu().numpy()
    ref = oracle.matvec(OKIND[kind], None, g, rows=rows, transpose=True)
    err = (np.abs(atg[:, rows] - ref).max(axis=1) / np.abs(g).sum(axis=1)).max()
    assert err <= TOL[prec], err


def _jac_tail_oracle(alpha, params, tail):
    """Rows j >= tail[0] of the reflection chain, exactly: upper triangularity means they only
    involve coefficients k >= tail[0] at every step."""
    a, b, g, d = params
    n = alpha.shape[-1]
    sign = (-1.0) ** np.arange(n)
    out = []
    for v in np.atleast_2d(alpha):
        y = np.zeros(n)
        y[tail] = sign[tail] * oracle.matvec(oracle.JAC, (b, a, d), sign * v, rows=tail)
        out.append(oracle.matvec(oracle.JAC, (a, d, g), y, rows=tail))
    return np.array(out)


@pytest.mark.parametrize("prec,tol,n", [("fp32", 1e-13, 70000), ("fp64", 1e-15, 40000)])
def test_jacobi_multipass(tdh, prec, tol, n):
    params = (0.1, -0.3, 0.0, 0.0)
    torch = _torch()
    alpha = workloads.coefficients(n, 2, decay=1.5, seed=5)
    plan = tdh.Plan("jac2jac", n, prec=prec, tol=tol, params=params)
    y = plan.execute(torch.tensor(alpha, dtype=plan.dtype, device="cuda")).double().cpu().numpy()
    tail = np.arange(n - 1500, n)
    ref = _jac_tail_oracle(alpha, params, tail)
    err = (np.abs(y[:, tail] - ref).max(axis=1) / np.abs(alpha).sum(axis=1)).max()
    assert err <= TOL[prec], err
    # prefix: alpha supported on [0, 4096) converts like the n = 4096 problem, zeros above
    a2 = alpha.copy()
    a2[:, 4096:] = 0.0
    y2 = plan.execute(torch.tensor(a2, dtype=plan.dtype, device="cuda")).double().cpu().numpy()
    ref2 = np.stack([oracle.jac2jac(v[:4096], *params) for v in a2])
    err = (np.abs(y2[:, :4096] - ref2).max(axis=1) / np.abs(a2).sum(axis=1)).max()
    assert err <= TOL[prec], err
    assert np.abs(y2[:, 4096:]).max() <= TOL[prec] * np.abs(a2).sum(axis=1).max()


def test_config4_jacobi_n2p20_b16(tdh):
    """P^(0.1,-0.3) -> P^(0,0), n = 2^20, batch 16, float32 execute, float64 plan, tol 1e-13:
    the last 1024 rows of every vector exactly against the oracle chain, and the prefix
    property on two vectors."""
    torch = _torch()
    n, batch = 1 << 20, 16
    params = (0.1, -0.3, 0.0, 0.0)
    alpha = workloads.coefficients(n, batch, decay=1.5, seed=0)
    plan = tdh.Plan("jac2jac", n, prec="fp32", tol=1e-13, params=params)
    y = plan.execute(torch.tensor(alpha, dtype=torch.float32, device="cuda")).double().cpu().numpy()
    assert np.all(np.isfinite(y))
    tail = np.arange(n - 1024, n)
    ref = _jac_tail_oracle(alpha, params, tail)
    err = (np.abs(y[:, tail] - ref).max(axis=1) / np.abs(alpha).sum(axis=1)).max()
    assert err <= 5e-6, err
    a2 = alpha[:2].copy()
    a2[:, 8192:] = 0.0
    y2 = plan.execute(torch.tensor(a2, dtype=torch.float32, device="cuda")).double().cpu().numpy()
    ref2 = np.stack([oracle.jac2jac(v[:8192], *params) for v in a2])
    err = (np.abs(y2[:, :8192] - ref2).max(axis=1) / np.abs(a2).sum(axis=1)).max()
    assert err <= 5e-6, err


@pytest.mark.parametrize("kind,params,prec", [
    ("jac2jac", (0.1, -0.3, 0.0, -0.3), "fp32"),
    ("jac2jac", (0.1, -0.3, 0.0, -0.3), "fp64"),
    ("leg2cheb", None, "fp32"),
], ids=["jacobi-fp32", "jacobi-fp64", "leg2cheb-fp32"])
def test_multipass_middle_rows_n2p20(tdh, kind, params, prec):
    """A single Case-2 step at n = 2^20 (multi-pass FFTs: 2^21 points in 256 slices for the
    rank-pair-packed Jacobi step, 2^20 in 128 for Legendre -> Chebyshev), batch 2, against the
    dense oracle on 320 rows spread over the whole vector: rows in the middle of every slice
    and of the cross-slice exchange, not only the tail."""
    torch = _torch()
    n, batch = 1 << 20, 2
    alpha = workloads.coefficients(n, batch, decay=1.5, seed=31)
    tol = 5e-6 if prec == "fp32" else 1e-12
    plan = tdh.Plan(kind, n, prec=prec, params=params or ())
    y = plan.execute(torch.tensor(alpha, dtype=plan.dtype, device="cuda")).double().cpu().numpy()
    rng = np.random.default_rng(32)
    rows = np.unique(np.r_[np.arange(32), n - 1 - np.arange(32), rng.integers(0, n, 256)])
    if kind == "jac2jac":
        ref = oracle.matvec(oracle.JAC, params[:3], alpha, rows=rows)
    else:
        ref = oracle.matvec(oracle.LEG2CHEB, None, alpha, rows=rows)
    err = (np.abs(y[:, rows] - ref).max(axis=1) / np.abs(alpha).sum(axis=1)).max()
    assert err <= tol, (err, plan.K)


def test_config4_supplementary_ultraspherical_case2_n2p20(tdh):
    """C^(0.25) -> C^(1.0) (Case 2, the Toeplitz-dot-Hankel path) at the config-4 size."""
    n, batch = 1 << 20, 16
    plan, alpha, y = _run(tdh, "ultra2ultra", n, batch, "fp32", 1e-13, decay=1.5, params=(0.25, 1.0))
    rows = _rows(n, k=48)
    ref = oracle.matvec(oracle.ULTRA, (0.25, 1.0), alpha, rows=rows)
    err = (np.abs(y[:, rows] - ref).max(axis=1) / np.abs(alpha).sum(axis=1)).max()
    assert err <= 5e-6, err


def test_jacobi_chebyshev_weight_equals_cheb2leg(tdh):
    """T_k = P_k^(-1/2,-1/2) / P_k^(-1/2,-1/2)(1) (Sec. 5.3): Jacobi (-1/2,-1/2) -> (0,0) of
    c_k / P_k(1) equals Chebyshev -> Legendre of c (two different plans, same answer)."""
    torch = _torch()
    n = 3000
    c = workloads.coefficients(n, 2, decay=1.0, seed=9)
    hi, _ = oracle.lambda_dd(2 * n + 2)
    pk1 = hi[2 * np.arange(n)] / np.sqrt(np.pi)  # P_k^(-1/2,-1/2)(1) = Lambda(k)/sqrt(pi)
    pj = tdh.Plan("jac2jac", n, prec="fp64", tol=1e-17, params=(-0.5, -0.5, 0.0, 0.0))
    pc = tdh.Plan("cheb2leg", n, prec="fp64", tol=1e-17)
    yj = pj.execute(torch.tensor(c / pk1, device="cuda")).cpu().numpy()
    yc = pc.execute(torch.tensor(c, device="cuda")).cpu().numpy()
    assert _rel_err(yj, yc, c) <= 1e-12


# ------------------------------------------------------------------------------- Laguerre

@pytest.mark.parametrize("params", [(0.5, -0.25), (0.3, 1.7), (2.0, 0.0), (0.0, 2.0)],
                         ids=["d=0.75", "d=-1.4", "d=2", "d=-2"])
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_laguerre(tdh, params, prec):
    """Sec. 5.4: a pure Toeplitz conversion (H all ones, rank 1).  Tolerance relative to the
    largest Toeplitz entry, which grows like m^(d-1)."""
    n = 3000
    tol = 1e-15 if prec == "fp64" else 1e-7
    plan, alpha, y = _run(tdh, "lag2lag", n, 2, prec, tol, decay=1.0, params=params)
    assert plan.K == 1
    ref = oracle.matvec(oracle.LAG, params, alpha)
    t = oracle.split(oracle.LAG, params, n)[0]
    scale = max(1.0, np.abs(t).max())
    assert _rel_err(y, ref, alpha) <= TOL[prec] * scale


def test_launch_count(tdh):
    """tdh_launch_count counts the kernels an execute call enqueues (one execute kernel, plus
    the balanced-split fix-up when vectors are split between clusters)."""
    torch = _torch()
    plan = tdh.Plan("leg2cheb", 1000, prec="fp32")
    x = torch.zeros(3, 1000, device="cuda")
    c0 = tdh.launch_count()
    plan.execute(x)
    torch.cuda.synchronize()
    assert 1 <= tdh.launch_count() - c0 <= 2


@pytest.mark.parametrize("batch", [1, 5, 35, 36, 37, 71, 144])
def test_balanced_split_batches(tdh, batch):
    """Batches below, at and above the number of resident clusters (36 four-CTA clusters on
    GB300): vectors split between clusters are summed by the fix-up in cluster order, and
    vectors owned whole by one cluster are written directly; every vector is checked."""
    torch = _torch()
    n = 65536
    alpha = workloads.coefficients(n, batch, decay=0.5, seed=21)
    plan = tdh.Plan("cheb2leg", n, prec="fp32", tol=1e-10)
    y = plan.execute(torch.tensor(alpha, dtype=torch.float32, device="cuda"))
    torch.cuda.synchronize()
    y = y.double().cpu().numpy()
    rows = np.unique(np.r_[np.arange(8), n - 1 - np.arange(8),
                           np.random.default_rng(22).integers(0, n, 16)])
    ref = oracle.matvec(oracle.CHEB2LEG, None, alpha, rows=rows)
    err = (np.abs(y[:, rows] - ref).max(axis=1) / np.abs(alpha).sum(axis=1)).max()
    assert err <= TOL["fp32"]
    # deterministic: the same call gives the same bits
    y2 = plan.execute(torch.tensor(alpha, dtype=torch.float32, device="cuda")).double().cpu().numpy()
    assert np.array_equal(y, y2)


@pytest.mark.parametrize("n,batch,pinned", [(65536, 100, True), (65537, 70, False), (1000, 3, True)],
                         ids=["chunks_pinned", "odd_n_pageable", "one_chunk"])
def test_execute_host_buffers(tdh, n, batch, pinned):
    """tdh_plan_execute_host: host vectors pass through the device in overlapped chunks; the
    result matches the device-buffer call (the chunks split the batch differently, so the two
    agree to rounding) and the oracle; the adjoint too."""
    torch = _torch()
    plan = tdh.Plan("leg2cheb", n, prec="fp32", tol=1e-7)
    alpha = workloads.coefficients(n, batch, decay=0.5, seed=23)
    x = torch.tensor(alpha, dtype=torch.float32)
    if pinned:
        x = x.pin_memory()
    y = plan.execute(x)
    g = plan.adjoint(x)
    torch.cuda.synchronize()
    assert y.device.type == "cpu" and g.device.type == "cpu"
    yd = plan.execute(x.cuda()).cpu()
    gd = plan.adjoint(x.cuda()).cpu()
    scale = np.abs(alpha).sum(axis=1).max()
    assert float((y - yd).abs().max()) <= 1e-6 * scale
    assert float((g - gd).abs().max()) <= 1e-6 * scale
    rows = np.unique(np.r_[np.arange(8), n - 1 - np.arange(8)])
    ref = oracle.matvec(oracle.LEG2CHEB, None, alpha[[0, batch - 1]], rows=rows)
    got = y.double().numpy()[[0, batch - 1]][:, rows]
    assert (np.abs(got - ref).max(axis=1) / np.abs(alpha[[0, batch - 1]]).sum(axis=1)).max() <= TOL["fp32"]


def test_largest_supported_length_and_beyond(tdh):
    """The largest float32 Legendre -> Chebyshev length, n = 2^23 (an FFT of 2^23 points: 512
    slices of 16384, the multi-pass path with the general cross stage), against the oracle on
    sampled rows; one coefficient more needs 2^24 points and is refused with UNSUPPORTED."""
    torch = _torch()
    n = 1 << 23
    alpha = workloads.coefficients(n, 1, decay=0.5, seed=24)
    plan = tdh.Plan("leg2cheb", n, prec="fp32", tol=1e-7)
    y = plan.execute(torch.tensor(alpha, dtype=torch.float32, device="cuda"))
    torch.cuda.synchronize()
    rows = np.unique(np.r_[np.arange(32), n - 1 - np.arange(32),
                           np.random.default_rng(25).integers(0, n, 64)])
    ref = oracle.matvec(oracle.LEG2CHEB, None, alpha, rows=rows)
    got = y.double().cpu().numpy()[:, rows]
    assert (np.abs(got - ref).max() / np.abs(alpha).sum()) <= TOL["fp32"]
    del plan, y
    with pytest.raises(tdh.TdhError) as e:
        tdh.Plan("leg2cheb", n + 1, prec="fp32", tol=1e-7)
    assert e.value.code == -2
