"""Independent polynomial machinery for pinning the oracle (no use of the paper's formulas).

Exact: each family's monomial coefficients from its three-term recurrence (DLMF 18.9) in
rational arithmetic, and the exact conversion matrix by back-substitution in the
monomial basis.  Floating point: Clenshaw summation of an expansion at a point.
"""
from fractions import Fraction as Fr

import numpy as np


def _poly_add(a, b):
    n = max(len(a), len(b))
    return [(a[i] if i < len(a) else 0) + (b[i] if i < len(b) else 0) for i in range(n)]


def _poly_scale(a, c):
    return [c * v for v in a]


def _poly_shift(a):  # multiply by x
    return [Fr(0)] + list(a)


def family(name, n, *params):
    """Monomial coefficients (lowest degree first) of phi_0..phi_{n-1}, exact rationals.

    name: 'legendre' | 'chebyshev' | 'gegenbauer'(lam) | 'jacobi'(a, b) | 'laguerre'(a).
    Parameters must be Fractions (or ints) for exactness.
    """
    polys = [[Fr(1)]]
    if n == 1:
        return polys
    for k in range(0, n - 1):
        A, B, C = recurrence(name, k, *params)
        nxt = _poly_add(_poly_add(_poly_scale(_poly_shift(polys[k]), A), _poly_scale(polys[k], B)),
                        _poly_scale(polys[k - 1], -C) if k >= 1 else [Fr(0)])
        polys.append(nxt[: k + 2])
    return polys


def recurrence(name, k, *params):
    """(A_k, B_k, C_k) with phi_{k+1} = (A_k x + B_k) phi_k - C_k phi_{k-1}, phi_0 = 1."""
    if name == "legendre":
        return Fr(2 * k + 1, k + 1), Fr(0), Fr(k, k + 1)
    if name == "chebyshev":
        return (Fr(1) if k == 0 else Fr(2)), Fr(0), Fr(1)
    if name == "gegenbauer":
        (lam,) = params
        return 2 * (k + lam) / Fr(k + 1), Fr(0), (k + 2 * lam - 1) / Fr(k + 1)
    if name == "jacobi":
        a, b = params
        if k == 0:
            return (a + b + 2) / Fr(2), (a - b) / Fr(2), Fr(0)
        s = 2 * k + a + b
        D = 2 * (k + 1) * (k + a + b + 1) * s
        return (s + 1) * (s + 2) * s / D, (s + 1) * (a * a - b * b) / D, 2 * (k + a) * (k + b) * (s + 2) / D
    if name == "laguerre":
        (a,) = params
        return Fr(-1, k + 1), (2 * k + 1 + a) / Fr(k + 1), (k + a) / Fr(k + 1)
    raise ValueError(name)


def conversion(src, dst):
    """Exact A with src_k = sum_j A[j][k] dst_j (dst_j of exact degree j)."""
    n = len(src)
    A = [[Fr(0)] * n for _ in range(n)]
    for k in range(n):
        p = list(src[k]) + [Fr(0)] * (n - len(src[k]))
        for j in range(k, -1, -1):
            c = p[j] / dst[j][j]
            A[j][k] = c
            if c:
                for i in range(j + 1):
                    p[i] -= c * dst[j][i]
    return A


def to_float(A):
    return np.array([[float(v) for v in row] for row in A])


def clenshaw(coef, x, name, *params):
    """sum_k coef[k] phi_k(x) by Clenshaw's backward recurrence, float64."""
    coef = np.asarray(coef, dtype=np.float64)
    n = coef.size
    rec = [tuple(float(v) for v in recurrence(name, k, *params)) for k in range(n + 1)]
    b1 = np.zeros_like(np.asarray(x, dtype=np.float64))
    b2 = np.zeros_like(b1)
    for k in range(n - 1, -1, -1):
        A, B, _ = rec[k]
        C_next = rec[k + 1][2]
        b0 = coef[k] + (A * x + B) * b1 - C_next * b2
        b2, b1 = b1, b0
    return b1
