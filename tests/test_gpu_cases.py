"""Integer and larger-than-one parameter differences (needs a GPU): Sec. 5.2 Cases 1 and 3
downward, Sec. 5.3 Cases 1 and 4 (sparse factors, their inverses by back-substitution, and
chains that end in a Case 2 / 3 step), and the Jacobi <-> Chebyshev conversions of Sec. 5.3's
end, against the dense oracle (whose closed forms are pinned by exact rationals).

Every check is max|beta - beta_ref| <= tol ||alpha||_1 kappa with the stated tolerances
(float64 1e-12, float32 5e-6) and the conversion's conditioning factor kappa
(tests/conditioning.py): 1 for conversions that raise every parameter (their outputs stay
below ||alpha||_1), so the stated bound holds as is; otherwise the output's own size
||beta_ref||_inf / ||alpha||_1, and for conversions with a Toeplitz-dot-Hankel step also the
largest entry max|A_jk|, in proportion to which the fast product errs.  Plans are
accuracy-targeted at half the stated tolerance.  Ultraspherical 20.5 -> 0.5 produces
coefficients near 1e102, beyond float32: float64 only.
"""
import numpy as np
import pytest

import oracle
import workloads
from conditioning import case1_only, kappa, output_kappa

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-12, "fp32": 5e-6}


@pytest.fixture(scope="module")
def tdh():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1604_07486_gb300 as m
    from paper_1604_07486_gb300 import build
    build.build()
    return m


def _err(y, ref, alpha):
    """max|y - ref| / ||alpha||_1 over the batch."""
    return (np.abs(y - ref).max(axis=-1) / np.abs(alpha).sum(axis=-1)).max()


def _bound(kind, params, prec, alpha=None, ref=None):
    """tol kappa: the stated tolerance times the conversion's conditioning factor (the
    output's own size, and for conversions with a Toeplitz-dot-Hankel step also the largest
    entry of the matrix), per unit of ||alpha||_1."""
    out = output_kappa(alpha, ref) if ref is not None else 1.0
    if case1_only(kind, params):
        return TOL[prec] * out
    return TOL[prec] * max(out, kappa(kind, tuple(params)))


def _execute(tdh, kind, params, alpha, prec, adjoint=False):
    """Accuracy-targeted plan at half the stated tolerance (each Toeplitz-dot-Hankel step's
    truncation), the default of the Python binding."""
    import torch
    plan = tdh.Plan(kind, alpha.shape[-1], prec=prec, tol=0.5 * TOL[prec], target=True,
                    params=params)
    x = torch.tensor(alpha, dtype=plan.dtype, device="cuda")
    y = plan.adjoint(x) if adjoint else plan.execute(x)
    torch.cuda.synchronize()
    return plan, y.double().cpu().numpy()


JAC = [
    ((0.5, 0.25, 1.5, 0.25), "case1_up"),
    ((1.5, 0.25, 0.5, 0.25), "case1_down"),
    ((0.5, 0.25, 3.5, 0.25), "case1_three_up"),
    ((0.25, 0.0, 1.75, 0.0), "case4_up"),
    ((1.75, 0.5, -0.5, 0.5), "case4_down"),
    ((0.625, -0.875, -0.75, -0.875), "case4_down_to_case3"),
    ((0.1, -0.3, 2.1, 1.7), "integer_both_parameters"),
    ((2.0, 1.5, -0.5, -0.25), "case4_both_parameters"),
    ((0.1, -0.3, 0.1, 1.7), "integer_b_reflected_only"),
    ((0.3, 2.6, 1.9, -0.2), "a_up_b_down"),
    ((1.5, 0.25, -0.5, -0.5), "to_chebyshev_weight"),
]


@pytest.mark.parametrize("params,name", JAC, ids=[c[1] for c in JAC])
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("n", [5001, 20000])
def test_jacobi_cases_1_4(tdh, params, name, prec, n):
    alpha = workloads.coefficients(n, 2, decay=1.5, seed=11)
    plan, y = _execute(tdh, "jac2jac", params, alpha, prec)
    rows = None if n <= 8192 else np.unique(np.r_[np.arange(64), n - 1 - np.arange(64),
                                                  np.random.default_rng(2).integers(0, n, 96)])
    ref = np.stack([oracle.jac2jac(v, *params, rows=rows) for v in alpha])
    yy = y if rows is None else y[:, rows]
    bound = _bound("jac2jac", params, prec, alpha, ref)
    assert _err(yy, ref, alpha) <= bound, (_err(yy, ref, alpha), bound, plan.K)


ULTRA = [((1.25, 0.25), "case1_down"), ((3.25, 0.25), "case1_three_down"),
         ((2.25, 0.75), "case3_down"), ((1.25, 0.5), "case2_down"),
         ((0.5, 20.5), "case1_twenty_up"), ((20.5, 0.5), "case1_twenty_down"),
         ((0.3, 18.1), "case3_eighteen_up")]


@pytest.mark.parametrize("params,name", ULTRA, ids=[c[1] for c in ULTRA])
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_ultraspherical_downward_and_long_chains(tdh, params, name, prec):
    """More than 16 whole steps take several sparse steps, the later ones in place (tile halos
    saved first); downward steps solve by back-substitution (tiled scan)."""
    if prec == "fp32" and name == "case1_twenty_down":
        pytest.skip("coefficients near 1e102 are beyond float32")
    n = 9001
    alpha = workloads.coefficients(n, 3, decay=1.5, seed=12)
    plan, y = _execute(tdh, "ultra2ultra", params, alpha, prec)
    ref = oracle.matvec(oracle.ULTRA, params, alpha)
    bound = _bound("ultra2ultra", params, prec, alpha, ref)
    assert _err(y, ref, alpha) <= bound, (_err(y, ref, alpha), bound, plan.K)


CHEB = [(0.25, -1 / 3), (1.5, 0.25), (-0.5, -0.5), (0.5, -0.5), (0.0, 0.0), (2.25, 1.0)]


@pytest.mark.parametrize("ab", CHEB, ids=[f"{a:g},{b:g}" for a, b in CHEB])
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_jac2cheb_cheb2jac(tdh, ab, prec):
    """T_k = P_k^(-1/2,-1/2) / P_k^(-1/2,-1/2)(1): the normalisation folds into the last
    (jac2cheb) or first (cheb2jac) step of the Jacobi chain."""
    n = 6000
    a, b = ab
    alpha = workloads.coefficients(n, 2, decay=1.5, seed=13)
    _, y = _execute(tdh, "jac2cheb", ab, alpha, prec)
    ref = np.stack([oracle.jac2cheb(v, a, b) for v in alpha])
    assert _err(y, ref, alpha) <= _bound("jac2cheb", ab, prec)
    _, y = _execute(tdh, "cheb2jac", ab, alpha, prec)
    ref = np.stack([oracle.cheb2jac(v, a, b) for v in alpha])
    assert _err(y, ref, alpha) <= _bound("cheb2jac", ab, prec)


def test_jac2cheb_legendre_equals_leg2cheb(tdh):
    """Jacobi (0, 0) is Legendre: jac2cheb(0, 0) reproduces the Legendre-to-Chebyshev plan."""
    import torch
    n = 3000
    alpha = workloads.coefficients(n, 2, decay=1.0, seed=14)
    _, y = _execute(tdh, "jac2cheb", (0.0, 0.0), alpha, "fp64")
    ref = oracle.matvec(oracle.LEG2CHEB, None, alpha)
    assert _err(y, ref, alpha) <= 1e-12


ADJ = [("ultra2ultra", (0.25, 2.25)), ("ultra2ultra", (3.25, 0.25)),
       ("ultra2ultra", (2.25, 0.75)), ("ultra2ultra", (0.25, 1.75)),
       ("jac2jac", (0.5, 0.25, 2.5, 0.25)), ("jac2jac", (1.75, 0.5, -0.5, 0.5)),
       ("jac2jac", (0.1, -0.3, 2.1, 1.7)), ("jac2jac", (2.0, 1.5, -0.5, -0.25)),
       ("jac2cheb", (0.25, 1.5)), ("cheb2jac", (1.5, 0.25))]


def _jac_T(g, a, b, c, d):
    """(Jacobi (a, b) -> (c, d))^T g: the oracle's chain transposed step by step."""
    if b == d and a == c:
        return g.copy()
    if b == d:
        return oracle.matvec(oracle.JAC, (a, b, c), g, transpose=True)
    sign = (-1.0) ** np.arange(g.shape[-1])
    y = g if a == c else oracle.matvec(oracle.JAC, (a, d, c), g, transpose=True)
    return sign * oracle.matvec(oracle.JAC, (b, a, d), sign * y, transpose=True)


def _transpose_ref(kind, params, g):
    if kind == "ultra2ultra":
        return oracle.matvec(oracle.ULTRA, params, g, transpose=True)
    if kind == "jac2jac":
        return _jac_T(g, *params)
    s = oracle.chebyshev_normalisation(g.shape[-1])
    a, b = params
    if kind == "jac2cheb":  # (diag(s) J)^T g = J^T (s g)
        return _jac_T(s * g, a, b, -0.5, -0.5)
    return _jac_T(g, -0.5, -0.5, a, b) / s  # (J diag(1/s))^T g


@pytest.mark.parametrize("kind,params", ADJ, ids=[f"{k}{p}" for k, p in ADJ])
def test_adjoint_against_transpose(tdh, kind, params):
    """A^T through the chain (steps reversed, sparse factors transposed, inverses run
    upward) equals the oracle's transpose; n spans several scan and sparse tiles."""
    n = 5000
    g = workloads.cotangent(n, 2, seed=15)
    ref = _transpose_ref(kind, params, g)
    # A^T has the same largest entry as A
    _, atg = _execute(tdh, kind, params, g, "fp64", adjoint=True)
    assert _err(atg, ref, g) <= _bound(kind, params, "fp64", g, ref)
    _, atg32 = _execute(tdh, kind, params, g, "fp32", adjoint=True)
    assert _err(atg32, ref, g) <= _bound(kind, params, "fp32", g, ref)


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_back_substitution_n2p20_b16(tdh, prec):
    """C^(1.25) -> C^(0.25) at n = 2^20, batch 16 (256 scan tiles per vector): sampled rows
    against the oracle."""
    n, batch = 1 << 20, 16
    alpha = workloads.coefficients(n, batch, decay=1.5, seed=16)
    _, y = _execute(tdh, "ultra2ultra", (1.25, 0.25), alpha, prec)
    rows = np.unique(np.r_[np.arange(64), n - 1 - np.arange(64),
                           np.random.default_rng(9).integers(0, n, 256)])
    ref = oracle.matvec(oracle.ULTRA, (1.25, 0.25), alpha, rows=rows)
    assert _err(y[:, rows], ref, alpha) <= _bound("ultra2ultra", (1.25, 0.25), prec, alpha, ref)


@pytest.mark.parametrize("n", [1, 2, 3, 4, 5, 4095, 4096, 4097, 8193])
def test_sparse_edge_lengths(tdh, n):
    """Short vectors and tile boundaries of both sparse kernels, upward and downward."""
    alpha = workloads.coefficients(n, 3, decay=1.0, seed=17)
    for params in [(0.5, 0.25, 1.5, 0.25), (1.5, 0.25, 0.5, 0.25)]:
        for prec in ("fp64", "fp32"):
            _, y = _execute(tdh, "jac2jac", params, alpha, prec)
            ref = np.stack([oracle.jac2jac(v, *params) for v in alpha])
            assert _err(y, ref, alpha) <= _bound("jac2jac", params, prec, alpha, ref), (params, prec)
