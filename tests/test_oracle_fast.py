"""The fast algorithm of Fig. 1 in float64 (oracle.fast_matvec, the CPU timing reference)
against the dense Direct product (oracle.matvec), for every single-step kind.

The difference has two parts: the truncation of the Hankel factorisation, at most
B(K) ||alpha||_1 (the PSD-residual bound of oracle.truncation_bound), and float64 rounding
of the FFTs, a few ulp of the largest intermediate times the scalings.  The pin therefore
asks max|beta_fast - beta| <= (B(K) + 1e-13) ||alpha||_1 at n <= 2000, and checks that a
planted slip in the fast product (a dropped rank term, the symbol's spectrum not
conjugated, a missing row-0 fix-up) breaks it.
"""
import numpy as np
import pytest

import oracle
import workloads

CASES = [
    ("leg2cheb", oracle.LEG2CHEB, None),
    ("cheb2leg", oracle.CHEB2LEG, None),
    ("ultra_up", oracle.ULTRA, (0.25, 0.75)),
    ("ultra_down", oracle.ULTRA, (1.25, 0.5)),
    ("jacobi_case2", oracle.JAC, (0.1, -0.3, 0.0)),
    ("jacobi_case3", oracle.JAC, (-0.7, -0.4, 0.2)),
    ("laguerre", oracle.LAG, (0.5, -0.25)),
]


def _err(y, ref, alpha):
    return (np.abs(y - ref).max(axis=-1) / np.abs(alpha).sum(axis=-1)).max()


@pytest.mark.parametrize("name,kind,params", CASES, ids=[c[0] for c in CASES])
@pytest.mark.parametrize("n", [257, 2000])
def test_fast_matvec_matches_dense_within_truncation_bound(name, kind, params, n):
    alpha = workloads.coefficients(n, 3, decay=1.0, seed=21)
    ref = oracle.matvec(kind, params, alpha)
    for target in (1e-6, 1e-12):
        plan = oracle.fast_plan(kind, params, n, target=target)
        bound = oracle.truncation_bound(kind, params, n, plan["u"])[-1]
        assert bound <= max(target, 1e-11)  # above target only at the rounding floor
        y = oracle.fast_apply(plan, alpha)
        assert _err(y, ref, alpha) <= bound + 1e-13, (target, len(plan["u"]))


def test_fast_matvec_relative_tolerance_and_workers():
    n = 1500
    alpha = workloads.coefficients(n, 2, decay=0.5, seed=22)
    ref = oracle.matvec(oracle.LEG2CHEB, None, alpha)
    y = oracle.fast_matvec(oracle.LEG2CHEB, None, alpha, tol=1e-15)
    assert _err(y, ref, alpha) <= 1e-13
    plan = oracle.fast_plan(oracle.LEG2CHEB, None, n, tol=1e-15)
    assert np.allclose(oracle.fast_apply(plan, alpha, workers=2), y, rtol=0, atol=1e-14)


def test_planted_slips_are_caught():
    n = 600
    alpha = workloads.coefficients(n, 2, decay=1.0, seed=23)
    for kind, params in ((oracle.LEG2CHEB, None), (oracle.CHEB2LEG, None)):
        ref = oracle.matvec(kind, params, alpha)
        plan = oracle.fast_plan(kind, params, n, target=1e-12)
        tol = oracle.truncation_bound(kind, params, n, plan["u"])[-1] + 1e-13
        assert _err(oracle.fast_apply(plan, alpha), ref, alpha) <= tol
        dropped = dict(plan, u=plan["u"][1:])
        assert _err(oracle.fast_apply(dropped, alpha), ref, alpha) > 1e3 * tol
        unconj = dict(plan, spec=np.conj(plan["spec"]))
        assert _err(oracle.fast_apply(unconj, alpha), ref, alpha) > 1e3 * tol
        if plan["row0"] is not None:
            norow = dict(plan, row0=None)
            assert _err(oracle.fast_apply(norow, alpha), ref, alpha) > 1e3 * tol
