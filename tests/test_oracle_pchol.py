"""Pins of the oracle's pivoted Cholesky (Sec. 2.1, Fig. 2) and of the pins' own teeth."""
import os
from fractions import Fraction as Fr

import numpy as np
import pytest

import oracle
import polys

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
EPS = np.finfo(np.float64).eps


def _H(kind, params, n):
    _, h, _, _ = oracle.split(kind, params, n)
    return oracle.hankel(h, n, oracle.first_index(kind))


def _golden_rank():
    vals = {}
    with open(os.path.join(GOLDEN, "pchol_rank_leg2cheb_N300.txt")) as f:
        for line in f:
            line = line.split("#")[0].strip()
            if line:
                k, v = line.split()
                vals[k] = int(v)
    return vals["N"], vals["K"]


def test_rank_at_N300_reaches_double_precision_within_paper_steps():
    """Sec. 2.1: 27 pivots give an approximant of the N = 300 Hankel part accurate to double
    precision.  The paper does not state its stop threshold; under any threshold between
    1e-16 and 1e-15 relative to max diag(H) the algorithm stops at no more than 27 steps,
    the residual is then at the rounding level, and 20 steps are still clearly short."""
    N, K_paper = _golden_rank()
    H = _H(oracle.LEG2CHEB, None, N + 1)
    for tol in (1e-15, EPS, 1e-16):
        ells, a, piv = oracle.pivoted_cholesky(lambda p: H[:, p], np.diag(H), tol)
        K = len(a)
        assert K_paper - 5 <= K <= K_paper, (tol, K)
        R = H - (ells.T / a) @ ells
        assert np.abs(R).max() <= 8 * EPS * np.abs(H).max()
    ells, a, _ = oracle.pivoted_cholesky(lambda p: H[:, p], np.diag(H), 0.0, kmax=20)
    R = H - (ells.T / a) @ ells
    assert np.abs(R).max() > 1e-14 * np.abs(H).max()


@pytest.mark.parametrize("kind,params", [(oracle.LEG2CHEB, None), (oracle.CHEB2LEG, None),
                                         (oracle.ULTRA, (0.75, 1.25)), (oracle.JAC, (0.1, -0.3, 0.0))])
def test_matches_full_update_form(kind, params):
    """The O(K^2 N) column form (Fig. 2, reading of its inner update) equals the O(K N^2)
    full-update form, Eq. (6): same pivots, same columns."""
    H = _H(kind, params, 200)
    e1, a1, p1 = oracle.pivoted_cholesky(lambda p: H[:, p], np.diag(H), 1e-14)
    e2, a2, p2 = oracle.pivoted_cholesky_full(H, 1e-14)
    K = min(len(a1), len(a2))
    assert K >= 10 and abs(len(a1) - len(a2)) <= 1
    assert np.array_equal(p1[:K], p2[:K])
    scale = np.abs(H).max()
    assert np.abs(e1[:K] - e2[:K]).max() <= 1e-12 * scale


def test_near_best_against_svd():
    """Fig. 3 (left): at N = 1000 the Cholesky approximants track the best rank-K
    approximants.  On the log scale of the figure the two errors fall by 15 orders of
    magnitude together; their ratio to sigma_{K+1} stays bounded at every rank."""
    H = _H(oracle.LEG2CHEB, None, 1001)
    sig = np.linalg.svd(H, compute_uv=False)
    ells, a, _ = oracle.pivoted_cholesky(lambda p: H[:, p], np.diag(H), 0.0, kmax=26)
    errs = []
    for K in range(1, 27):
        err = np.linalg.norm(H - (ells[:K].T / a[:K]) @ ells[:K], 2)
        assert sig[K] * (1 - 1e-6) <= err <= 60 * sig[K], (K, err, sig[K])
        errs.append(err)
    assert errs[-1] < 1e-13 * errs[0]


def test_rank_grows_like_log_N():
    """Thm 3.5: K = O(log N log 1/eps).  At fixed tol, multiplying N by 256 adds a bounded
    number of pivots rather than multiplying K."""
    Ks = []
    for n in (256, 4096, 65536):
        u, _ = oracle.hankel_factors(oracle.LEG2CHEB, None, n, 1e-15)
        Ks.append(len(u))
    assert Ks[0] < Ks[1] < Ks[2]
    assert Ks[2] - Ks[1] <= 12 and Ks[1] - Ks[0] <= 12
    assert Ks[2] < 2 * Ks[0]


@pytest.mark.parametrize("kind,params", [(oracle.LEG2CHEB, None), (oracle.CHEB2LEG, None)])
def test_residual_bounded_by_tolerance(kind, params):
    """PSD residual: |R_jk| <= sqrt(d_j d_k) <= tol * max diag(H) at the stop."""
    n = 700
    H = _H(kind, params, n)
    tol = 1e-10
    u, _ = oracle.hankel_factors(kind, params, n, tol)
    j0 = oracle.first_index(kind)
    R = H - u[:, j0:].T @ u[:, j0:]
    assert np.abs(R).max() <= 2 * tol * np.diag(H).max()


# ------------------------------------------------------------ the pins have teeth

def test_garbled_update_is_rejected():
    """Taken literally, Fig. 2's printed update l_r <- l_r - l_j (l_r)_j / (l_r)_{p_r} does
    not reproduce Eq. (6); the comparison above would catch it."""
    H = _H(oracle.LEG2CHEB, None, 120)
    d = np.diag(H).copy()
    ells, piv = [], []
    with np.errstate(invalid="ignore", divide="ignore"):  # the literal form divides by 0
        for _ in range(8):
            p = int(np.argmax(d))
            ell = H[:, p].copy()
            for j in range(len(ells)):
                ell = ell - ells[j] * ell[j] / ell[p]
            ells.append(ell)
            piv.append(p)
            d = d - ell * ell / ell[p]
    e2, a2, p2 = oracle.pivoted_cholesky_full(H, 0.0, kmax=8)
    assert not (np.array_equal(np.array(piv), p2) and np.allclose(np.array(ells), e2, atol=1e-12))


@pytest.mark.parametrize("mutation", ["transpose", "row0_factor", "sign", "shift"])
def test_exact_pin_catches_planted_mistakes(mutation):
    """Plausible mistakes in the closed form (a transposed operand, the row-0 factor of
    Eq. (2) dropped, a sign flip, an index shift) fail the exact-rational comparison."""
    n = 12
    exact = polys.to_float(polys.conversion(polys.family("legendre", n), polys.family("chebyshev", n)))
    A = oracle.entries(oracle.LEG2CHEB, None, n)
    if mutation == "transpose":
        A = A.T
    elif mutation == "row0_factor":
        A = A.copy()
        A[0] *= 2.0
    elif mutation == "sign":
        A = -A
    elif mutation == "shift":
        A = np.roll(A, 1, axis=1)
    assert np.abs(A - exact).max() > 1e-3
