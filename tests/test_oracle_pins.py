"""Pins of the CPU oracle against facts the paper and the mathematics fix (no GPU).

Each test checks the oracle against something other than itself: exact rational
conversion matrices built from the polynomial recurrences (DLMF 18.9), Clenshaw
evaluation of both expansions, L M = I, the Hankel moment integrals, the Gamma-ratio
special values, and an mpmath evaluation of Lambda.
"""
from fractions import Fraction as Fr
import os

import numpy as np
import pytest

import oracle
import polys

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")

# (oracle kind, params, source family, target family) with exact rational parameters
CASES = [
    ("leg2cheb", oracle.LEG2CHEB, None, ("legendre",), ("chebyshev",)),
    ("cheb2leg", oracle.CHEB2LEG, None, ("chebyshev",), ("legendre",)),
    ("ultra_case2", oracle.ULTRA, (0.75, 1.25), ("gegenbauer", Fr(3, 4)), ("gegenbauer", Fr(5, 4))),
    ("ultra_case2_down", oracle.ULTRA, (1.25, 0.5), ("gegenbauer", Fr(5, 4)), ("gegenbauer", Fr(1, 2))),
    ("ultra_case1", oracle.ULTRA, (0.25, 1.25), ("gegenbauer", Fr(1, 4)), ("gegenbauer", Fr(5, 4))),
    ("ultra_case1_two", oracle.ULTRA, (0.25, 2.25), ("gegenbauer", Fr(1, 4)), ("gegenbauer", Fr(9, 4))),
    ("jac_case2", oracle.JAC, (0.1, -0.3, 0.0), ("jacobi", Fr(1, 10), Fr(-3, 10)), ("jacobi", Fr(0), Fr(-3, 10))),
    ("jac_case2_paper", oracle.JAC, (0.0, 0.5, -0.25), ("jacobi", Fr(0), Fr(1, 2)), ("jacobi", Fr(-1, 4), Fr(1, 2))),
    ("jac_to_cheb", oracle.JAC, (0.0, -0.5, -0.5), ("jacobi", Fr(0), Fr(-1, 2)), ("jacobi", Fr(-1, 2), Fr(-1, 2))),
    ("jac_case1", oracle.JAC, (0.5, 0.25, 1.5), ("jacobi", Fr(1, 2), Fr(1, 4)), ("jacobi", Fr(3, 2), Fr(1, 4))),
    ("jac_case3_cheb", oracle.JAC, (-0.5, -0.5, 0.25), ("jacobi", Fr(-1, 2), Fr(-1, 2)), ("jacobi", Fr(1, 4), Fr(-1, 2))),
    ("jac_case3", oracle.JAC, (-0.6, -0.7, -0.2), ("jacobi", Fr(-3, 5), Fr(-7, 10)), ("jacobi", Fr(-1, 5), Fr(-7, 10))),
    ("lag", oracle.LAG, (0.5, -0.25), ("laguerre", Fr(1, 2)), ("laguerre", Fr(-1, 4))),
    # integer and larger-than-one differences: the same closed forms (Sec. 5.2 Cases 1/3,
    # Sec. 5.3 Cases 1/4), downward and upward
    ("ultra_case1_down", oracle.ULTRA, (1.25, 0.25), ("gegenbauer", Fr(5, 4)), ("gegenbauer", Fr(1, 4))),
    ("ultra_case3_down", oracle.ULTRA, (2.25, 0.75), ("gegenbauer", Fr(9, 4)), ("gegenbauer", Fr(3, 4))),
    ("jac_case1_down", oracle.JAC, (1.5, 0.25, 0.5), ("jacobi", Fr(3, 2), Fr(1, 4)), ("jacobi", Fr(1, 2), Fr(1, 4))),
    ("jac_case1_two", oracle.JAC, (0.5, 0.25, 2.5), ("jacobi", Fr(1, 2), Fr(1, 4)), ("jacobi", Fr(5, 2), Fr(1, 4))),
    ("jac_case4_up", oracle.JAC, (0.25, 0.0, 1.75), ("jacobi", Fr(1, 4), Fr(0)), ("jacobi", Fr(7, 4), Fr(0))),
    ("jac_case4_down", oracle.JAC, (1.75, 0.5, -0.5), ("jacobi", Fr(7, 4), Fr(1, 2)), ("jacobi", Fr(-1, 2), Fr(1, 2))),
    ("jac_case4_to_case3", oracle.JAC, (0.625, -0.875, -0.75), ("jacobi", Fr(5, 8), Fr(-7, 8)), ("jacobi", Fr(-3, 4), Fr(-7, 8))),
]


def _exact(src, dst, n):
    return polys.conversion(polys.family(src[0], n, *src[1:]), polys.family(dst[0], n, *dst[1:]))


@pytest.mark.parametrize("name,kind,params,src,dst", CASES, ids=[c[0] for c in CASES])
def test_entries_match_exact_conversion(name, kind, params, src, dst):
    """Closed-form entries (Eqs. (2), (11), (13), Sec. 5.3, 5.4) equal the
    exact conversion matrix from the polynomial recurrences, to a few ulp."""
    n = 12
    exact = polys.to_float(_exact(src, dst, n))
    A = oracle.entries(kind, params, n)
    scale = np.maximum(np.abs(exact), 1e-300)
    assert np.all(np.abs(A - exact) <= 4e-16 * scale + 1e-300), np.abs(A - exact).max()
    # the sparsity of the exact matrix is reproduced (zeros where k - j is odd, etc.)
    assert np.array_equal(exact == 0.0, A == 0.0)


@pytest.mark.parametrize("name,kind,params,src,dst", [c for c in CASES if c[1] != oracle.LAG],
                         ids=[c[0] for c in CASES if c[1] != oracle.LAG])
def test_split_identity(name, kind, params, src, dst):
    """A = D1 (T o H) D2 with the paper's split (Eq. (7), Sec. 5.1-5.3)
    reproduces the exact matrix; for Chebyshev-to-Legendre on indices j, k >= 1 only,
    since Sec. 5.1 applies row 0 directly."""
    n = 12
    exact = polys.to_float(_exact(src, dst, n))
    t, h, d1, d2 = oracle.split(kind, params, n)
    j = np.arange(n)[:, None]
    k = np.arange(n)[None, :]
    T = np.where(k >= j, t[np.clip(k - j, 0, n - 1)], 0.0)
    A = d1[:, None] * T * h[j + k] * d2[None, :]
    j0 = oracle.first_index(kind, params)
    sub = (slice(j0, n), slice(j0, n))
    assert np.allclose(A[sub], exact[sub], rtol=2e-15, atol=1e-300)


def test_worked_constants():
    """P_2 = 3/4 T_2 + 1/4 T_0 gives M_00 = 1, M_11 = 1, M_02 = 1/4, M_22 = 3/4 (Eq. (2));
    T_2 = 4/3 P_2 - 1/3 P_0 gives L_02 = -1/3, L_22 = 4/3 (Eq. (11))."""
    vals = {}
    with open(os.path.join(GOLDEN, "worked_entries.txt")) as f:
        for line in f:
            line = line.split("#")[0].strip()
            if line:
                key, num, den = line.split()
                vals[key] = int(num) / int(den)
    M = oracle.entries(oracle.LEG2CHEB, None, 4)
    L = oracle.entries(oracle.CHEB2LEG, None, 4)
    for key, v in vals.items():
        mat = M if key[0] == "M" else L
        j, k = int(key[1]), int(key[2])
        assert abs(mat[j, k] - v) <= 2e-16 * abs(v)


def test_inverse_pair():
    """L = M^{-1} (Sec. 5.1)."""
    n = 96
    M = oracle.entries(oracle.LEG2CHEB, None, n)
    L = oracle.entries(oracle.CHEB2LEG, None, n)
    assert np.abs(L @ M - np.eye(n)).max() < 1e-13
    assert np.abs(M @ L - np.eye(n)).max() < 1e-13


def test_identity_cases():
    """lambda1 = lambda2 and (a, b) = (g, d) give the identity; Jacobi (0,0) is Legendre, so
    Jacobi (0,0) -> (-1/2,-1/2) equals Legendre-to-Chebyshev up to the normalisation
    T_k = P_k^(-1/2,-1/2) / P_k^(-1/2,-1/2)(1) (Sec. 5.3)."""
    n = 40
    assert np.abs(oracle.entries(oracle.ULTRA, (0.7, 0.7), n) - np.eye(n)).max() < 1e-15
    assert np.abs(oracle.entries(oracle.JAC, (0.3, -0.2, 0.3), n) - np.eye(n)).max() < 1e-14
    x = np.random.default_rng(3).standard_normal(n)
    # P^(0,0) -> P^(-1/2,-1/2) through the reflection chain, then rescale to T_k
    y = oracle.jac2jac(x, 0.0, 0.0, -0.5, -0.5)
    kk = np.arange(n)
    # P_k^(-1/2,-1/2)(1) = Gamma(k+1/2)/(Gamma(1/2) k!) = Lambda(k)/sqrt(pi)
    lam_hi, lam_lo = oracle.lambda_dd(2 * n + 2)
    pk1 = lam_hi[2 * kk] / np.sqrt(np.pi)
    cheb = y * pk1
    ref = oracle.matvec(oracle.LEG2CHEB, None, x)
    assert np.abs(cheb - ref).max() < 1e-13 * np.abs(x).sum()


@pytest.mark.parametrize("kind,params,src,dst", [
    (oracle.LEG2CHEB, None, ("legendre",), ("chebyshev",)),
    (oracle.CHEB2LEG, None, ("chebyshev",), ("legendre",)),
    (oracle.ULTRA, (0.75, 1.25), ("gegenbauer", 0.75), ("gegenbauer", 1.25)),
    (oracle.ULTRA, (0.25, 1.25), ("gegenbauer", 0.25), ("gegenbauer", 1.25)),
    (oracle.JAC, (0.1, -0.3, 0.0), ("jacobi", 0.1, -0.3), ("jacobi", 0.0, -0.3)),
])
def test_clenshaw_evaluation(kind, params, src, dst):
    """Both expansions of the same polynomial agree at random points in [-1, 1]."""
    n = 700
    rng = np.random.default_rng(11)
    a = rng.standard_normal(n) / (np.arange(n) + 1.0)
    b = oracle.matvec(kind, params, a)
    x = rng.uniform(-1, 1, 64)
    p = polys.clenshaw(a, x, *src)
    q = polys.clenshaw(b, x, *dst)
    assert np.abs(p - q).max() < 1e-12 * np.abs(a).sum()


def test_jacobi_reflection_chain_exact():
    """beta != delta: the reflection chain of Sec. 5.3 reproduces the exact direct conversion
    P^(1/10,-3/10) -> P^(0,0) built from the recurrences (no chaining on the exact side)."""
    n = 12
    exact = polys.to_float(_exact(("jacobi", Fr(1, 10), Fr(-3, 10)), ("jacobi", Fr(0), Fr(0)), n))
    A = np.stack([oracle.jac2jac(e, 0.1, -0.3, 0.0, 0.0) for e in np.eye(n)], axis=1)
    assert np.abs(A - exact).max() < 1e-14 * np.abs(exact).max()


def test_lambda_special_values_and_mpmath():
    """Lambda(0) = sqrt(pi), Lambda(1/2) = 2/sqrt(pi); the double-double table matches mpmath
    at 40 digits, including large arguments where log-gamma differences lose accuracy."""
    mpmath = pytest.importorskip("mpmath")
    mpmath.mp.dps = 40
    count = (1 << 17) + 3
    hi, lo = oracle.lambda_dd(count)
    sp = mpmath.sqrt(mpmath.pi)
    assert abs(mpmath.mpf(hi[0]) + mpmath.mpf(lo[0]) - sp) < mpmath.mpf(10) ** -30
    assert abs(mpmath.mpf(hi[1]) + mpmath.mpf(lo[1]) - 2 / sp) < mpmath.mpf(10) ** -30
    for i in [2, 3, 17, 1000, 4097, 65535, 65536, count - 1]:
        z = mpmath.mpf(i) / 2
        ref = mpmath.gamma(z + mpmath.mpf(1) / 2) / mpmath.gamma(z + 1)
        got = mpmath.mpf(hi[i]) + mpmath.mpf(lo[i])
        assert abs(got / ref - 1) < mpmath.mpf(10) ** -26, (i, got, ref)


def _gauss_jacobi_01(npts, a, b):
    """Nodes/weights for int_0^1 f(x) x^b (1-x)^a dx via scipy's Gauss-Jacobi rule."""
    from scipy.special import roots_jacobi
    t, w = roots_jacobi(npts, a, b)  # weight (1-t)^a (1+t)^b on [-1, 1]
    x = (t + 1) / 2
    return x, w / 2 ** (a + b + 1)


def test_hankel_moment_integrals():
    """The Hankel generators are moments of the measures the paper gives (Thm 3.2, Sec. 5.1,
    5.2, Eq. (15)); evaluated by Gauss-Jacobi quadrature, not Gamma ratios."""
    from math import gamma, pi, sqrt
    n = 40
    s = np.arange(2 * n - 1)
    # Leg->Cheb: h_s = 2/sqrt(pi) int_0^1 x^s (1-x^2)^(-1/2) dx, weight (1-x)^(-1/2),
    # smooth factor x^s (1+x)^(-1/2)
    x, w = _gauss_jacobi_01(80, -0.5, 0.0)
    ref = np.array([2 / sqrt(pi) * (w * x ** si * (1 + x) ** -0.5).sum() for si in s])
    _, h, _, _ = oracle.split(oracle.LEG2CHEB, None, n)
    assert np.allclose(h, ref, rtol=1e-13)
    # Cheb->Leg (s >= 2): h_s = 4/sqrt(pi) int_0^1 x^(s-1) (1-x^2)^(1/2) dx
    x, w = _gauss_jacobi_01(80, 0.5, 0.0)
    ref = np.array([4 / sqrt(pi) * (w * x ** (si - 1) * (1 + x) ** 0.5).sum() for si in s[2:]])
    _, h, _, _ = oracle.split(oracle.CHEB2LEG, None, n)
    assert np.allclose(h[2:], ref, rtol=1e-13)
    # ultraspherical: h_s = 2 G(l2)/(G(l1) G(l2-l1+1)) int_0^1 x^(s+2 l1-1) (1-x^2)^(l2-l1) dx
    l1, l2 = 0.75, 1.25
    x, w = _gauss_jacobi_01(80, l2 - l1, 2 * l1 - 1)
    c = 2 * gamma(l2) / (gamma(l1) * gamma(l2 - l1 + 1))
    ref = np.array([c * (w * x ** si * (1 + x) ** (l2 - l1)).sum() for si in s])
    _, h, _, _ = oracle.split(oracle.ULTRA, (l1, l2), n)
    assert np.allclose(h, ref, rtol=1e-12)
    # Jacobi: H_jk proportional to int_0^1 x^(j+k) x^(a+b) (1-x)^(g-a) dx
    a, b, g = 0.1, -0.3, 0.0
    x, w = _gauss_jacobi_01(80, g - a, a + b)
    mom = np.array([(w * x ** si).sum() for si in s])
    _, h, _, _ = oracle.split(oracle.JAC, (a, b, g), n)
    assert np.allclose(h / h[0], mom / mom[0], rtol=1e-12)


@pytest.mark.parametrize("kind,params", [(oracle.LEG2CHEB, None), (oracle.CHEB2LEG, None),
                                         (oracle.ULTRA, (0.75, 1.25)), (oracle.JAC, (0.1, -0.3, 0.0)),
                                         (oracle.JAC, (-0.6, -0.7, -0.2))])
def test_hankel_psd(kind, params):
    """The Hankel part is positive semidefinite (on indices >= 1 for Chebyshev-to-Legendre and
    Jacobi Case 3, Sec. 5.1 and 5.3)."""
    n = 160
    _, h, _, _ = oracle.split(kind, params, n)
    H = oracle.hankel(h, n, oracle.first_index(kind, params))
    ev = np.linalg.eigvalsh(H)
    assert ev.min() > -1e-14 * ev.max()


def test_adjoint_matches_transpose():
    """matvec(transpose=True) applies A^T: <A x, g> = <x, A^T g> and the dense transpose."""
    n = 300
    rng = np.random.default_rng(5)
    x = rng.standard_normal(n)
    g = rng.standard_normal(n)
    for kind, params in [(oracle.LEG2CHEB, None), (oracle.CHEB2LEG, None), (oracle.JAC, (0.1, -0.3, 0.0))]:
        A = oracle.entries(kind, params, n)
        ax = oracle.matvec(kind, params, x)
        atg = oracle.matvec(kind, params, g, transpose=True)
        assert np.allclose(ax, A @ x, rtol=0, atol=1e-13 * np.abs(x).sum() * np.abs(A).max())
        assert np.allclose(atg, A.T @ g, rtol=0, atol=1e-13 * np.abs(g).sum() * np.abs(A).max())
        assert abs(ax @ g - x @ atg) < 1e-12 * np.abs(ax).sum() * np.abs(g).max()


def test_sampled_rows_equal_dense():
    n = 500
    x = np.random.default_rng(2).standard_normal((3, n))
    rows = np.array([0, 1, 7, 250, 499])
    full = oracle.matvec(oracle.CHEB2LEG, None, x)
    part = oracle.matvec(oracle.CHEB2LEG, None, x, rows=rows)
    assert np.array_equal(full[:, rows], part)


@pytest.mark.parametrize("a,b", [(Fr(1, 4), Fr(-1, 3)), (Fr(0), Fr(-1, 2)), (Fr(3, 2), Fr(1, 4)),
                                 (Fr(-1, 2), Fr(-1, 2))])
def test_jac2cheb_cheb2jac_exact(a, b):
    """Jacobi <-> Chebyshev through T_k = P_k^(-1/2,-1/2) / P_k^(-1/2,-1/2)(1) (Sec. 5.3, end)
    equals the exact conversion between the two families built from their recurrences."""
    n = 12
    exact_jc = polys.to_float(_exact(("jacobi", a, b), ("chebyshev",), n))
    exact_cj = polys.to_float(_exact(("chebyshev",), ("jacobi", a, b), n))
    I = np.eye(n)
    A = np.stack([oracle.jac2cheb(e, float(a), float(b)) for e in I], axis=1)
    B = np.stack([oracle.cheb2jac(e, float(a), float(b)) for e in I], axis=1)
    assert np.abs(A - exact_jc).max() < 2e-14 * np.abs(exact_jc).max()
    assert np.abs(B - exact_cj).max() < 2e-14 * np.abs(exact_cj).max()


def _bidiagonal(n, off, diag, sup):
    S = [[Fr(0)] * n for _ in range(n)]
    for j in range(n):
        S[j][j] = diag(j)
        if j + off < n:
            S[j][j + off] = sup(j)
    return S


def test_sparse_factor_readings():
    """The sparse factors the GPU path applies for integer steps, checked exactly.

    Sec. 5.2, Eq. (12): (S_l)_jj = l/(l+j), (S_l)_{j,j+2} = -l/(l+j+2) maps
    C^(l) coefficients to C^(l+1) coefficients.  Sec. 5.3 Case 1: S_(a,b) maps (a, b)
    coefficients to (a+1, b) coefficients with diagonal (j+a+b+1)/(2j+a+b+1) (1 at j = 0)
    and superdiagonal -(j+b+1)/(2j+a+b+3).  The paper prints the superdiagonal numerator
    as j+a+1, which is the factor for raising b instead (up to sign); the exact conversion
    decides for j+b+1, and the printed form fails whenever a != b."""
    n = 10
    for lam in (Fr(1, 4), Fr(3, 2)):
        S = _bidiagonal(n, 2, lambda j: lam / (lam + j), lambda j: -lam / (lam + j + 2))
        exact = _exact(("gegenbauer", lam), ("gegenbauer", lam + 1), n)
        assert S == exact
    for a, b in ((Fr(1, 2), Fr(1, 4)), (Fr(-1, 2), Fr(-3, 4)), (Fr(1, 3), Fr(1, 3))):
        s = a + b
        diag = lambda j: Fr(1) if j == 0 else (j + s + 1) / (2 * j + s + 1)
        S = _bidiagonal(n, 1, diag, lambda j: -(j + b + 1) / (2 * j + s + 3))
        exact = _exact(("jacobi", a, b), ("jacobi", a + 1, b), n)
        assert S == exact
        printed = _bidiagonal(n, 1, diag, lambda j: -(j + a + 1) / (2 * j + s + 3))
        assert (printed == exact) == (a == b)
        # raising b: the reflection P_k^(a,b)(x) = (-1)^k P_k^(b,a)(-x) flips the
        # superdiagonal's sign
        Sb = _bidiagonal(n, 1, diag, lambda j: (j + a + 1) / (2 * j + s + 3))
        assert Sb == _exact(("jacobi", a, b), ("jacobi", a, b + 1), n)
