"""Pins of the accuracy-targeted truncation bound (oracle.truncation_bound, target_rank).

The bound rests on one fact about the pivoted Cholesky of Sec. 2.1 (Fig. 2): the residual
R = H - sum_{r<K} u_r u_r^T of a positive semidefinite H is positive semidefinite, so
|R_jk| <= sqrt(d_j d_k).  Through A = D1 (T o H) D2 (Eq. (3)) every entry
of A - A_K is then at most max|t| |d1_j| sqrt(d_j) |d2_k| sqrt(d_k).  These tests check the
bound against the dense error of every prefix, by brute force on small n, and show that
plausible slips in writing it down are caught.
"""
import numpy as np
import pytest

import oracle

EPS = np.finfo(np.float64).eps

KINDS = [(oracle.LEG2CHEB, None), (oracle.CHEB2LEG, None), (oracle.ULTRA, (0.75, 1.25)),
         (oracle.ULTRA, (1.5, 0.7)), (oracle.JAC, (0.1, -0.3, 0.0)), (oracle.JAC, (-0.4, 0.25, 0.35))]


def _dense_errors(kind, params, n, u):
    """max |A - A_K'| over the Hankel block for every prefix K' of u (dense, float64)."""
    t, h, d1, d2 = oracle.split(kind, params, n)
    j0 = oracle.first_index(kind, params)
    A = oracle.entries(kind, params, n)
    j = np.arange(n)
    T = np.where(j[None, :] >= j[:, None], t[np.abs(j[None, :] - j[:, None])], 0.0)
    errs, scale = [], np.abs(A[j0:, j0:]).max()
    for k in range(len(u) + 1):
        G = u[:k].T @ u[:k]
        Ak = d1[:, None] * T * G * d2[None, :]
        errs.append(np.abs(A[j0:, j0:] - Ak[j0:, j0:]).max())
    return np.array(errs), scale


def _mutated_bound(kind, params, n, u, mutation):
    t, h, d1, d2 = oracle.split(kind, params, n)
    j0 = oracle.first_index(kind, params)
    d = np.zeros(n)
    d[j0:] = h[2 * np.arange(j0, n)]
    out = []
    for k in range(len(u) + 1):
        dd = np.maximum(d, 0.0)
        if mutation == "d_not_sqrt":
            s = dd
        else:
            s = np.sqrt(dd)
        if mutation == "one_diagonal":
            b = np.abs(t).max() * np.max(np.abs(d1) * s) * np.max(s)
        elif mutation == "residual_off_by_one":
            b = None
        else:
            b = np.abs(t).max() * np.max(np.abs(d1) * s) * np.max(np.abs(d2) * s)
        out.append(b)
        if k < len(u):
            d = d - u[k] * u[k]
    if mutation == "residual_off_by_one":  # bound of K' reported for K' - 1 terms
        good = oracle.truncation_bound(kind, params, n, u)
        return np.r_[good[1:], good[-1]]
    return np.array(out)


@pytest.mark.parametrize("weighted", [False, True])
@pytest.mark.parametrize("kind,params", KINDS)
def test_bound_dominates_dense_error(kind, params, weighted):
    """Every prefix: max |A - A_K'| <= B(K') (up to the rounding of the dense product), for
    the factors of H and for those of the congruent W H W (pivot weights), converted back."""
    n = 56
    w = oracle.pivot_weights(kind, params, n) if weighted else None
    u, _ = oracle.hankel_factors(kind, params, n, 1e-18, kmax=n, weights=w)
    b = oracle.truncation_bound(kind, params, n, u)
    errs, scale = _dense_errors(kind, params, n, u)
    assert len(b) == len(u) + 1 and len(u) >= 8
    slack = 64 * n * EPS * scale
    assert np.all(errs <= b * (1 + 1e-12) + slack), np.c_[errs, b][errs > b + slack]
    # not vacuous: the bound falls with the rank, to the rounding level
    assert b[-1] < 1e-12 * b[0]
    assert np.all(np.diff(b) <= 1e-12 * b[0])


@pytest.mark.parametrize("mutation", ["d_not_sqrt", "one_diagonal", "residual_off_by_one"])
def test_bound_pin_catches_planted_mistakes(mutation):
    """A bound written down wrongly (d for sqrt(d); D2 dropped; the residual of one term
    fewer) falls below the true dense error for some prefix and kind."""
    caught = False
    for kind, params in KINDS:
        n = 56
        u, _ = oracle.hankel_factors(kind, params, n, 1e-18, kmax=n)
        bad = _mutated_bound(kind, params, n, u, mutation)
        errs, scale = _dense_errors(kind, params, n, u)
        if np.any(errs > bad * (1 + 1e-12) + 64 * n * EPS * scale):
            caught = True
            break
    assert caught, mutation


@pytest.mark.parametrize("kind,params", [(oracle.LEG2CHEB, None), (oracle.CHEB2LEG, None)])
def test_target_rank_meets_target(kind, params):
    """target_rank: monotone in the target; the product with K' terms is within
    target * ||alpha||_1 of the exact one (dense, n = 400, random alpha)."""
    n = 400
    prev = -1
    rng = np.random.default_rng(7)
    alpha = rng.standard_normal((3, n)) / np.sqrt(np.arange(1, n + 1))
    t, h, d1, d2 = oracle.split(kind, params, n)
    j0 = oracle.first_index(kind, params)
    j = np.arange(n)
    T = np.where(j[None, :] >= j[:, None], t[np.abs(j[None, :] - j[:, None])], 0.0)
    A = oracle.entries(kind, params, n)
    u, _ = oracle.hankel_factors(kind, params, n, 1e-18, kmax=128,
                                 weights=oracle.pivot_weights(kind, params, n))
    for target in (1e-3, 1e-6, 1e-9, 1e-12):
        k, bound = oracle.target_rank(kind, params, n, target)
        assert k >= prev and bound <= target
        prev = k
        Ak = d1[:, None] * T * (u[:k].T @ u[:k]) * d2[None, :]
        Ak[:j0, :] = A[:j0, :]
        Ak[:, :j0] = A[:, :j0]
        err = np.abs(alpha @ (A - Ak).T).max(axis=1) / np.abs(alpha).sum(axis=1)
        assert err.max() <= target, (target, k, err.max())


def test_weighted_pivots_need_fewer_terms_for_chebyshev_to_legendre():
    """Chebyshev -> Legendre has D1 and D2 growing like j: pivoting on W H W (w = sqrt|D1 D2|)
    reaches a worst-case target with fewer terms than pivoting on H, and the weighted
    factors reproduce H as well as the unweighted ones at full rank."""
    n = 4096
    for target in (2.5e-6, 1e-8):
        kw, _ = oracle.target_rank(oracle.CHEB2LEG, None, n, target, weighted=True)
        ku, _ = oracle.target_rank(oracle.CHEB2LEG, None, n, target, weighted=False)
        assert kw < ku, (target, kw, ku)
    n = 300
    _, h, _, _ = oracle.split(oracle.CHEB2LEG, None, n)
    H = oracle.hankel(h, n, 1)
    u, _ = oracle.hankel_factors(oracle.CHEB2LEG, None, n, 1e-18, kmax=n,
                                 weights=oracle.pivot_weights(oracle.CHEB2LEG, None, n))
    assert np.abs(H - u[:, 1:].T @ u[:, 1:]).max() <= 1e-13 * np.abs(H).max()
