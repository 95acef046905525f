"""Conditioning factor of a conversion, for the accuracy checks of the GPU tests.

The fast product rounds relative to the norm of its whole input: a rank term's FFT error is
about u log2(L) ||t||_1 ||u_r o D2 alpha||_2 at every output index, then scaled by
|D1_j u_r[j]| (Eq. (5); the paper's own experiments show this error growing with N, Sec. 4,
Table 1).  When no entry of the conversion matrix exceeds 1 (every parameter raised, and the
Legendre/Chebyshev pair), that is a modest multiple of u ||alpha||_1 and the stated tolerance
tol ||alpha||_1 applies as is.  Lowering a parameter makes entries grow with the index, the
same rounding grows with them (normwise: u max|A_jk| ||alpha||_1), and the output itself can
exceed tol / u ||alpha||_1, past which even its own final rounding breaks tol ||alpha||_1.
The tests therefore check

    max |beta - beta_ref| <= tol ||alpha||_1 kappa,
    kappa = max(1, ||beta_ref||_inf / ||alpha||_1, max_{j,k < 512} |A_jk|)

for every conversion with a Toeplitz-dot-Hankel step.  Conversions made of Case-1 steps only
(integer parameter differences, Sec. 5.2, 5.3: banded factors and back-substitution) round
componentwise, not normwise; for them the only limit is the output's own rounding, and
kappa = max(1, ||beta_ref||_inf / ||alpha||_1) (see ``case1_only``).

A_jk does not depend on n (the n x n conversion is the leading block of any larger one), so
the largest entry of the leading 512 x 512 block is a lower bound of the largest entry at the
test's n: the check is at least as strict as tol ||alpha||_1 max(1, max|A_jk|).  The block is
computed exactly by the oracle (its dense product applied to the 512 unit vectors).
"""
import functools

import numpy as np

import oracle

KAPPA_N = 512


def _apply(kind, params, X):
    if kind == "ultra2ultra":
        return oracle.matvec(oracle.ULTRA, params, X)
    if kind == "jac2jac":
        return np.stack([oracle.jac2jac(v, *params) for v in X])
    if kind == "jac2cheb":
        return np.stack([oracle.jac2cheb(v, *params) for v in X])
    if kind == "cheb2jac":
        return np.stack([oracle.cheb2jac(v, *params) for v in X])
    if kind == "leg2cheb":
        return oracle.matvec(oracle.LEG2CHEB, None, X)
    if kind == "cheb2leg":
        return oracle.matvec(oracle.CHEB2LEG, None, X)
    raise ValueError(kind)


@functools.lru_cache(maxsize=None)
def kappa(kind, params=None):
    """max(1, max |A_jk|) over the leading KAPPA_N x KAPPA_N block of the conversion."""
    cols = _apply(kind, tuple(params) if params is not None else None, np.eye(KAPPA_N))
    return max(1.0, float(np.abs(cols).max()))


def _integer(x):
    return abs(x - round(x)) <= 1e-14 * max(1.0, abs(x))


def case1_only(kind, params):
    """True when every parameter difference is an integer: no Toeplitz-dot-Hankel step."""
    if kind == "ultra2ultra":
        return _integer(params[1] - params[0])
    if kind == "jac2jac":
        return _integer(params[2] - params[0]) and _integer(params[3] - params[1])
    return False


def output_kappa(alpha, beta_ref):
    """max(1, max over the batch of ||beta_ref||_inf / ||alpha||_1)."""
    a = np.abs(np.atleast_2d(alpha)).sum(axis=-1)
    b = np.abs(np.atleast_2d(beta_ref)).max(axis=-1)
    return max(1.0, float((b / a).max()))
