"""Plain CPU oracle for polynomial basis conversion (TEST INFRASTRUCTURE ONLY).

What the CUDA path is checked against.  Only tests/, __graft_entry__.smoke() and the
CPU-baseline legs of bench.py may import this module; the library never does.

Source: Townsend, Webb & Olver, "Fast polynomial transforms based on Toeplitz and Hankel
matrices" (arXiv:1604.07486).

* ``matvec`` / ``entries`` / ``split`` wrap the double-double C oracle (tdh_oracle.c):
  the dense "Direct" product of Sec. 4 with entries from their closed forms.
* ``pivoted_cholesky`` is the O(K^2 N) algorithm of Sec. 2.1 (Fig. 2), steps in the
  paper's order, in float64.  Reading of the garbled inner update of Fig. 2: step j is
  applied to the new column as l_r <- l_r - l_j (l_j)_{p_r} / a_j, which is what the
  prose of Sec. 2.1 describes (apply each earlier Cholesky step to column p_r).
* ``pivoted_cholesky_full`` is the O(K N^2) full-update form, Eq. (6).
* ``jac2jac`` composes the Case-2 formula with the reflection of Sec. 5.3 when
  beta != delta (reading: P_k^(a,b)(x) = (-1)^k P_k^(b,a)(-x)).  The closed form of
  Sec. 5.3 holds for every parameter pair (its Gamma ratios come from recurrences, which
  continue through integer differences), so the oracle takes no integer steps: Cases 1 and
  4 are the same formula.
* ``jac2cheb`` / ``cheb2jac`` use T_k = P_k^(-1/2,-1/2) / P_k^(-1/2,-1/2)(1) (Sec. 5.3,
  end): a Jacobi (-1/2, -1/2) conversion and a diagonal scaling.
* ``fast_plan`` / ``fast_apply`` / ``fast_matvec`` are the outline of Fig. 1 in float64
  with numpy's (or scipy's) FFT as the Toeplitz step: the CPU timing reference of the same
  algorithm, pinned against the dense ``matvec`` within the truncation bound; never the
  parity truth for the GPU path.
* ``truncation_bound`` / ``target_rank`` / ``pivot_weights``: the accuracy-targeted choice of
  the rank (a reading, not in the paper): the PSD residual of the Fig. 2 factorisation bounds
  every entry of A - A_K; the factorisation may pivot on W H W (w = sqrt|d1 d2|), the same A.
  Pinned against dense residuals by brute force (tests/test_oracle_truncation.py).
"""
import ctypes
import os

import numpy as np

from . import build as _build

LEG2CHEB, CHEB2LEG, ULTRA, JAC, LAG = 0, 1, 2, 3, 4

_lib = None


def _load():
    global _lib
    if _lib is None:
        path = _build.build()
        lib = ctypes.CDLL(path)
        i64, dbl_p, i64_p = ctypes.c_int64, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int64)
        lib.tdho_matvec.argtypes = [ctypes.c_int, dbl_p, i64, dbl_p, i64, i64, i64_p, i64, dbl_p,
                                    i64, ctypes.c_int, ctypes.c_int]
        lib.tdho_entries.argtypes = [ctypes.c_int, dbl_p, i64, i64, i64, i64, i64, dbl_p]
        lib.tdho_split.argtypes = [ctypes.c_int, dbl_p, i64, dbl_p, dbl_p, dbl_p, dbl_p]
        lib.tdho_lambda.argtypes = [i64, dbl_p, dbl_p]
        lib.tdho_threads.argtypes = []
        for f in (lib.tdho_matvec, lib.tdho_entries, lib.tdho_split, lib.tdho_lambda, lib.tdho_threads):
            f.restype = ctypes.c_int
        _lib = lib
    return _lib


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _params(params):
    p = np.zeros(4, dtype=np.float64)
    if params is not None:
        p[: len(params)] = params
    return p


def threads():
    """Host threads the dense oracle runs on."""
    return int(_load().tdho_threads())


def matvec(kind, params, x, rows=None, transpose=False, nthreads=0):
    """beta = A x (or A^T x) for every row in ``rows`` (all rows if None).

    x: float64 array [batch][n] or [n].  Returns float64 [batch][len(rows)] (or 1-D).
    """
    lib = _load()
    x = np.ascontiguousarray(x, dtype=np.float64)
    squeeze = x.ndim == 1
    if squeeze:
        x = x[None, :]
    batch, n = x.shape
    p = _params(params)
    if rows is None:
        nrows, rows_p = n, None
    else:
        rows = np.ascontiguousarray(rows, dtype=np.int64)
        nrows = rows.size
        rows_p = rows.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))
    y = np.zeros((batch, nrows), dtype=np.float64)
    rc = lib.tdho_matvec(kind, _dp(p), n, _dp(x), batch, n, rows_p, nrows, _dp(y), nrows,
                         1 if transpose else 0, nthreads)
    if rc != 0:
        raise ValueError(f"oracle matvec failed ({rc})")
    return y[0] if squeeze else y


def entries(kind, params, n, j0=0, j1=None, k0=0, k1=None):
    """Dense block A[j0:j1, k0:k1] from the closed forms (rounded once to float64)."""
    j1 = n if j1 is None else j1
    k1 = n if k1 is None else k1
    out = np.zeros((j1 - j0, k1 - k0), dtype=np.float64)
    rc = _load().tdho_entries(kind, _dp(_params(params)), n, j0, j1, k0, k1, _dp(out))
    if rc != 0:
        raise ValueError(f"oracle entries failed ({rc})")
    return out


def split(kind, params, n):
    """Generator sequences of A = D1 (T o H) D2: (t[n], h[2n-1], d1[n], d2[n])."""
    t = np.zeros(n)
    h = np.zeros(2 * n - 1)
    d1 = np.zeros(n)
    d2 = np.zeros(n)
    rc = _load().tdho_split(kind, _dp(_params(params)), n, _dp(t), _dp(h), _dp(d1), _dp(d2))
    if rc != 0:
        raise ValueError(f"oracle split failed ({rc})")
    return t, h, d1, d2


def lambda_dd(count):
    """Lambda(i/2) = Gamma(i/2 + 1/2)/Gamma(i/2 + 1), i < count, as (hi, lo) double-double."""
    hi = np.zeros(count)
    lo = np.zeros(count)
    _load().tdho_lambda(count, _dp(hi), _dp(lo))
    return hi, lo


def hankel(h, n, j0=0):
    """Dense Hankel block H[j, k] = h[j + k] for j, k in [j0, n)."""
    idx = np.arange(j0, n)
    return h[idx[:, None] + idx[None, :]]


def first_index(kind, params=None):
    """Index where the positive semidefinite Hankel block starts: row 0 is applied directly for
    Chebyshev-to-Legendre (Sec. 5.1) and for Jacobi Case 3, a + b <= -1 (Sec. 5.3)."""
    if kind == CHEB2LEG:
        return 1
    if kind == JAC and params is not None and params[0] + params[1] <= -1.0:
        return 1
    return 0


# ---------------------------------------------------------------- pivoted Cholesky

def pivoted_cholesky(column, diag, tol, kmax=None):
    """Sec. 2.1, Fig. 2: rank-K approximation H ~ sum_r l_r l_r^T / a_r.

    column(p) -> H[:, p] (float64, length N); diag = diag(H).
    Stops before step r once the pivot is negligible (Sec. 2.1): max(d) <= tol * d0
    or the pivot entry a_r = (l_r)_{p_r} of the updated column <= tol * d0, where
    d0 = max(diag(H)).  (a_r is the diagonal entry of H^(r-1) that d approximates; the
    two differ only by rounding, and checking both keeps a_r > 0.)
    Ties in the argmax go to the lowest index.  Returns (ells [K][N], a [K], pivots [K]).
    """
    d = np.array(diag, dtype=np.float64, copy=True)
    N = d.size
    kmax = N if kmax is None else min(kmax, N)
    d0 = float(d.max()) if N else 0.0
    ells, a, piv = [], [], []
    for _ in range(kmax):
        p = int(np.argmax(d))
        if not d[p] > tol * d0:
            break
        ell = np.array(column(p), dtype=np.float64, copy=True)
        for j in range(len(ells)):
            ell -= ells[j] * (ells[j][p] / a[j])
        a_r = float(ell[p])
        if not a_r > tol * d0:
            break
        ells.append(ell)
        a.append(a_r)
        piv.append(p)
        d -= ell * ell / a_r
    return np.array(ells).reshape(len(ells), N), np.array(a), np.array(piv, dtype=np.int64)


def pivoted_cholesky_full(H, tol, kmax=None):
    """Eq. (6) applied repeatedly: H^(r) = H^(r-1) - H_{:,p} H_{p,:} / H_pp.

    The O(K N^2) form that updates the whole matrix; same pivot and stop rule as
    ``pivoted_cholesky``.  Returns (ells, a, pivots) with l_r = H^(r-1)[:, p_r].
    """
    R = np.array(H, dtype=np.float64, copy=True)
    N = R.shape[0]
    kmax = N if kmax is None else min(kmax, N)
    d0 = float(np.diag(R).max()) if N else 0.0
    ells, a, piv = [], [], []
    for _ in range(kmax):
        dg = np.diag(R)
        p = int(np.argmax(dg))
        if not dg[p] > tol * d0:
            break
        col = R[:, p].copy()
        ells.append(col)
        a.append(float(col[p]))
        piv.append(p)
        R = R - np.outer(col, R[p, :]) / col[p]
    return np.array(ells).reshape(len(ells), N), np.array(a), np.array(piv, dtype=np.int64)


def pivot_weights(kind, params, n):
    """w_j = sqrt(|d1_j d2_j|) (1 where that is 0): the diagonal W of the congruence W H W
    on which an accuracy-targeted factorisation pivots.  W H W is positive semidefinite when
    H is, and A = D1 (T o H) D2 = (D1 W^-1) (T o W H W) (W^-1 D2)."""
    _, _, d1, d2 = split(kind, params, n)
    w = np.sqrt(np.abs(d1 * d2))
    w[~((w > 0) & np.isfinite(w))] = 1.0
    return w


def hankel_factors(kind, params, n, tol, kmax=None, weights=None):
    """Pivoted Cholesky of the PSD Hankel part of ``kind`` on indices [j0, n).

    Returns (u [K][n], pivots) with u_r = l_r / sqrt(a_r) zero-extended below j0, so that
    H[j0:, j0:] ~ sum_r u_r u_r^T.  With ``weights`` w the factorisation (Fig. 2, same steps)
    runs on W H W, entries w_j h_{j+k} w_k, and its factors are returned divided by w, so the
    same identity holds; only the pivots (and the stop) differ.
    """
    t, h, d1, d2 = split(kind, params, n)
    j0 = first_index(kind, params)
    idx = np.arange(j0, n)
    w = np.ones(len(idx)) if weights is None else np.asarray(weights, dtype=np.float64)[idx]
    ells, a, piv = pivoted_cholesky(lambda p: h[idx + idx[p]] * w * w[p], h[2 * idx] * w * w,
                                    tol, kmax)
    u = np.zeros((len(a), n))
    if len(a):
        u[:, j0:] = ells / np.sqrt(a)[:, None] / w
    return u, piv + j0


def truncation_bound(kind, params, n, u):
    """Bound on the entries of A - A_K for the rank-K factors u (from ``hankel_factors``),
    for every prefix K' = 0..K (array of K + 1 values).

    The residual R = H - sum_{r<K'} u_r u_r^T of a pivoted Cholesky of a positive
    semidefinite H is positive semidefinite, so each 2 x 2 principal minor gives
    |R_jk| <= sqrt(d_j d_k) with d = diag(R).  A - A_K' = D1 (T o R) D2 on the Hankel block
    (Sec. 2, Eq. (3)), hence
        |(A - A_K')_jk| <= max|t| * |d1_j| sqrt(d_j) * |d2_k| sqrt(d_k),
    and max_j |beta_K' - beta| <= B(K') ||alpha||_1 with
        B(K') = max|t| * max_j |d1_j| sqrt(d_j) * max_k |d2_k| sqrt(d_k).
    """
    t, h, d1, d2 = split(kind, params, n)
    j0 = first_index(kind, params)
    d = np.zeros(n)
    d[j0:] = h[2 * np.arange(j0, n)]
    tmax = np.abs(t).max()
    out = []
    for k in range(len(u) + 1):
        s = np.sqrt(np.maximum(d, 0.0))
        out.append(tmax * np.max(np.abs(d1) * s) * np.max(np.abs(d2) * s))
        if k < len(u):
            d = d - u[k] * u[k]
    return np.array(out)


def target_rank(kind, params, n, target, tol=1e-18, kmax=128, weighted=True):
    """Fewest rank terms K' whose ``truncation_bound`` is <= target, for the factors of a
    pivoted Cholesky run to relative tolerance ``tol`` (at most kmax steps) on W H W
    (``weighted``, w from ``pivot_weights``) or on H; all of them if no prefix meets the
    target.  Returns (K', bound at K').  The bound is the same expression for weighted
    factors: |D1_j / w_j| sqrt(w_j^2 d_j) = |D1_j| sqrt(d_j)."""
    w = pivot_weights(kind, params, n) if weighted else None
    u, _ = hankel_factors(kind, params, n, tol, kmax, weights=w)
    b = truncation_bound(kind, params, n, u)
    ok = np.nonzero(b <= target)[0]
    k = int(ok[0]) if len(ok) else len(u)
    return k, float(b[k])


# ---------------------------------------------------------------- compositions

def jac2jac(x, a, b, g, d, rows=None):
    """Jacobi (a, b) -> (g, d) coefficients.

    beta == delta: the Case-2 formula directly.  Otherwise (Sec. 5.3 reflection):
    flip signs, convert (b, a) -> (d, a), flip back, then convert (a, d) -> (g, d).
    """
    x = np.asarray(x, dtype=np.float64)
    if b == d and a == g:
        return x.copy() if rows is None else x[..., np.asarray(rows)].copy()
    if b == d:
        return matvec(JAC, (a, b, g), x, rows=rows)
    n = x.shape[-1]
    sign = (-1.0) ** np.arange(n)
    y = sign * matvec(JAC, (b, a, d), sign * x)
    if a == g:
        return y if rows is None else y[..., np.asarray(rows)]
    return matvec(JAC, (a, d, g), y, rows=rows)


def chebyshev_normalisation(n):
    """P_k^(-1/2,-1/2)(1) = Gamma(k + 1/2) / (Gamma(1/2) Gamma(k + 1)) = Lambda(k)/sqrt(pi),
    k < n (DLMF 18.6.1), from the double-double Lambda table."""
    hi, lo = lambda_dd(2 * n)
    return (hi[0::2] + lo[0::2]) / np.sqrt(np.pi)


def jac2cheb(x, a, b, rows=None):
    """Jacobi (a, b) -> Chebyshev: convert to Jacobi (-1/2, -1/2), then c_k <- c_k
    P_k^(-1/2,-1/2)(1), since P_k^(-1/2,-1/2) = P_k^(-1/2,-1/2)(1) T_k (Sec. 5.3, end)."""
    x = np.asarray(x, dtype=np.float64)
    s = chebyshev_normalisation(x.shape[-1])
    y = jac2jac(x, a, b, -0.5, -0.5, rows=rows)
    return y * (s if rows is None else s[np.asarray(rows)])


def cheb2jac(x, a, b, rows=None):
    """Chebyshev -> Jacobi (a, b): c_k <- c_k / P_k^(-1/2,-1/2)(1), then Jacobi
    (-1/2, -1/2) -> (a, b)."""
    x = np.asarray(x, dtype=np.float64)
    s = chebyshev_normalisation(x.shape[-1])
    return jac2jac(x / s, -0.5, -0.5, a, b, rows=rows)


# ---------------------------------------------------------------- fast product (Fig. 1)

def fast_plan(kind, params, n, tol=1e-15, target=None):
    """Steps 1-2 of Fig. 1 in float64 for vectors of n coefficients: the split (Eq. (3)),
    the Fig. 2 factors of H (relative tolerance ``tol``; or, with ``target``, the fewest terms
    of the weighted factorisation whose truncation bound is <= target), and the spectrum of
    the Toeplitz symbol for the zero-padded length L >= 2n - 1.  Row 0 of the Chebyshev-to-
    Legendre and Jacobi Case-3 products is kept for a direct dot product (Sec. 5.1, 5.3)."""
    t, h, d1, d2 = split(kind, params, n)
    if target is None:
        u, _ = hankel_factors(kind, params, n, tol)
    else:
        w = pivot_weights(kind, params, n)
        u, _ = hankel_factors(kind, params, n, 1e-18, 128, weights=w)
        ok = np.nonzero(truncation_bound(kind, params, n, u) <= target)[0]
        u = u[: int(ok[0]) if len(ok) else len(u)]
    L = 1
    while L < 2 * n - 1:
        L *= 2
    row0 = entries(kind, params, n, 0, 1)[0] if first_index(kind, params) == 1 else None
    return {"n": n, "L": L, "spec": np.conj(np.fft.rfft(t, L)), "u": u, "d1": d1, "d2": d2,
            "row0": row0}


def fast_apply(plan, x, workers=None):
    """Steps 3-5 of Fig. 1: v = D2 x; w = sum_r u_r o T (u_r o v), each Toeplitz product by a
    zero-padded real FFT of length L, multiplied by the conjugate spectrum of t (a
    correlation, since T_jk = t_{k-j}); beta = D1 w, then row 0 directly where the plan keeps
    it.  ``workers`` > 1 runs the FFTs on that many host threads (scipy.fft)."""
    x = np.atleast_2d(np.asarray(x, dtype=np.float64))
    n, L = plan["n"], plan["L"]
    if workers and workers > 1:
        import scipy.fft as sf
        rfft = lambda a: sf.rfft(a, L, axis=-1, workers=workers)
        irfft = lambda a: sf.irfft(a, L, axis=-1, workers=workers)
    else:
        rfft = lambda a: np.fft.rfft(a, L, axis=-1)
        irfft = lambda a: np.fft.irfft(a, L, axis=-1)
    v = x * plan["d2"]
    w = np.zeros_like(v)
    for ur in plan["u"]:
        w += ur * irfft(rfft(v * ur) * plan["spec"])[..., :n]
    beta = w * plan["d1"]
    if plan["row0"] is not None:
        beta[:, 0] = x @ plan["row0"]
    return beta


def fast_matvec(kind, params, x, tol=1e-15, target=None):
    """beta = A x by the fast algorithm of Fig. 1 in float64 (one Toeplitz-dot-Hankel step:
    Leg<->Cheb, ultraspherical and Jacobi Case 2/3, Laguerre).  A CPU timing reference,
    pinned against ``matvec`` within the truncation bound (tests/test_oracle_fast.py)."""
    x = np.atleast_2d(np.asarray(x, dtype=np.float64))
    return fast_apply(fast_plan(kind, params, x.shape[-1], tol, target), x)
