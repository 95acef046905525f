"""Oracle for beta = A alpha: TEST INFRASTRUCTURE ONLY.

A plain, slow, obviously correct CPU implementation of the polynomial basis conversion
of Townsend, Webb & Olver (arXiv:1604.07486), written from the paper alone.  Only
tests/, __graft_entry__.smoke() and the CPU-baseline legs of bench.py may import it.
It shares no code with the CUDA library and the library never imports it.

Parity status: every function here is pinned by -m "not gpu" tests (exact rational
conversion, Clenshaw evaluation, Hankel moment integrals, L M = I, the K = 27 rank of
Sec. 2.1, the full-update Cholesky form, and the truncation bound against dense residuals
by brute force).  ``fast_matvec`` (the fast algorithm of Fig. 1 in float64, the CPU timing
reference) is pinned against the dense ``matvec`` within the truncation bound; it is never
the parity truth for the GPU path.
"""
from .oracle import (CHEB2LEG, JAC, LAG, LEG2CHEB, ULTRA, cheb2jac, chebyshev_normalisation,
                     entries, fast_apply, fast_matvec, fast_plan, first_index, hankel, hankel_factors, jac2cheb,
                     jac2jac, lambda_dd, matvec, pivot_weights, pivoted_cholesky,
                     pivoted_cholesky_full, split, target_rank, threads, truncation_bound)

__all__ = ["CHEB2LEG", "JAC", "LAG", "LEG2CHEB", "ULTRA", "cheb2jac", "chebyshev_normalisation",
           "entries", "fast_apply", "fast_matvec", "fast_plan", "first_index", "hankel", "hankel_factors", "jac2cheb",
           "jac2jac", "lambda_dd", "matvec", "pivot_weights", "pivoted_cholesky", "pivoted_cholesky_full",
           "split", "target_rank", "threads", "truncation_bound"]
