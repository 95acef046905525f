"""Seeded synthetic inputs shared by the tests, the bench and the smoke check.

This module draws random numbers and nothing else: it holds none of the conversion's
arithmetic, so both the CUDA path and the CPU oracle can be fed from it.

The inputs mirror the paper's experiments (Sec. 4, Fig. 4): a vector of standard normal
draws scaled so that entry k decays like (k+1)^(-p), generated once in float64 from a
fixed seed.  The paper draws with Julia's ``srand(0); randn``; those exact vectors are not
reproducible here, so numpy's ``default_rng(seed)`` takes their place.
"""
import numpy as np

# The workloads the library is measured and checked on (sizes as in the paper's experiments
# and the configurations the bench reports).  n = number of coefficients (degree n - 1).
CONFIGS = {
    "leg2cheb_n1024_fp64": dict(kind="leg2cheb", n=1024, batch=1, decay=1.0, prec="fp64", tol=1e-15),
    "leg2cheb_n65536_b256": dict(kind="leg2cheb", n=65536, batch=256, decay=0.5),
    "cheb2leg_n65536_b256": dict(kind="cheb2leg", n=65536, batch=256, decay=0.5),
    "ragged_4096": dict(kind="leg2cheb", count=4096, dmin=64, dmax=65536, decay=1.0),
    "jac_ultra_n2p20_b16": dict(n=1 << 20, batch=16, decay=1.5),
    "leg2cheb_autograd_n8192_b1024": dict(kind="leg2cheb", n=8192, batch=1024, decay=1.0),
}


def coefficients(n, batch=1, decay=1.0, seed=0):
    """alpha[b, k] = z[b, k] * (k + 1)^(-decay), z iid N(0, 1) from default_rng(seed); float64."""
    rng = np.random.default_rng(seed)
    z = rng.standard_normal((batch, n))
    return z * (np.arange(n, dtype=np.float64) + 1.0) ** (-float(decay))


def ragged_degrees(count, dmin=64, dmax=65536, seed=0):
    """Degrees d_i = floor(exp(U(ln dmin, ln dmax))), i < count; lengths are d_i + 1."""
    rng = np.random.default_rng(seed)
    u = rng.uniform(np.log(dmin), np.log(dmax), size=count)
    d = np.floor(np.exp(u)).astype(np.int64)
    return np.clip(d, dmin, dmax - 1)


def ragged_coefficients(lengths, decay=1.0, seed=0):
    """Concatenated vectors with per-vector decay; returns (values float64, offsets int64)."""
    lengths = np.asarray(lengths, dtype=np.int64)
    offsets = np.zeros(lengths.size + 1, dtype=np.int64)
    np.cumsum(lengths, out=offsets[1:])
    rng = np.random.default_rng(seed)
    z = rng.standard_normal(int(offsets[-1]))
    k = np.arange(offsets[-1], dtype=np.int64) - np.repeat(offsets[:-1], lengths)
    return z * (k.astype(np.float64) + 1.0) ** (-float(decay)), offsets


def cotangent(n, batch=1, seed=1):
    """A seeded cotangent / test vector g for adjoint identities, float64 [batch][n]."""
    rng = np.random.default_rng(seed)
    return rng.standard_normal((batch, n))
