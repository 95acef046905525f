"""GB300 Toeplitz-dot-Hankel polynomial basis conversion (Townsend, Webb & Olver,
arXiv:1604.07486): beta = A alpha with A = D1 (T o H) D2, H compressed by pivoted Cholesky,
each Toeplitz product by FFT -- all in the CUDA library libtdh.so (include/tdh.h).

This module only marshals arguments to that C ABI.  PyTorch supplies device memory and
streams; every step of the conversion runs in the library's kernels.  There is no CPU
fallback: if the library is not built or no GPU is present, calls raise.
"""
import ctypes
import os

from . import build as _build

LEG2CHEB, CHEB2LEG, ULTRA2ULTRA, JAC2JAC, LAG2LAG, JAC2CHEB, CHEB2JAC = 0, 1, 2, 3, 4, 5, 6
FP64, FP32, BF16X3 = 0, 1, 2
KINDS = {"leg2cheb": LEG2CHEB, "cheb2leg": CHEB2LEG, "ultra2ultra": ULTRA2ULTRA,
         "jac2jac": JAC2JAC, "lag2lag": LAG2LAG, "jac2cheb": JAC2CHEB, "cheb2jac": CHEB2JAC}
PRECS = {"fp64": FP64, "fp32": FP32, "bf16x3": BF16X3}
ERRORS = {0: "OK", -1: "INVALID_ARG", -2: "UNSUPPORTED", -3: "NOMEM", -4: "ALIGN",
          -5: "TIMEOUT", -6: "CUDA", -7: "ALIAS"}

# Every entry point include/tdh.h declares (checked by the CPU test suite).
EXPORTS = ("tdh_plan_create", "tdh_plan_execute", "tdh_plan_execute_adjoint", "tdh_plan_query",
           "tdh_plan_destroy", "tdh_last_error", "tdh_symbols", "tdh_pchol", "tdh_pchol_noalloc",
           "tdh_plan_execute_ragged", "tdh_launch_count", "tdh_plan_execute_host",
           "tdh_plan_schedule_count", "tdh_plan_schedule_info", "tdh_plan_set_schedule",
           "tdh_plan_autotune", "tdh_schedules", "tdh_alloc_stats", "tdh_test_fail_alloc",
           "tdh_measure_fma_rate", "tdh_plan_status", "tdh_test_tc_stall",
           "tdh_plan_execute_ragged_host", "tdh_measure_dsmem_rate")
FLAG_RAGGED = 1
FLAG_TARGET = 2


class TdhError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{ERRORS.get(code, code)}: {msg}")
        self.code = code


class _Params(ctypes.Structure):
    _fields_ = [("p", ctypes.c_double * 4), ("prec", ctypes.c_int), ("flags", ctypes.c_int),
                ("kmax", ctypes.c_int64)]


_lib = None


def library_path():
    return _build.LIB


def lib():
    """Load libtdh.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        path = library_path()
        if not os.path.exists(path):
            raise RuntimeError(f"CUDA library not built ({path}); call "
                               "paper_1604_07486_gb300.build.build() first")
        L = ctypes.CDLL(path)
        vp, i64, dbl = ctypes.c_void_p, ctypes.c_int64, ctypes.c_double
        L.tdh_plan_create.argtypes = [ctypes.c_int, i64, ctypes.POINTER(_Params), dbl,
                                      ctypes.POINTER(vp)]
        L.tdh_plan_execute.argtypes = [vp, vp, vp, i64, vp]
        L.tdh_plan_execute_adjoint.argtypes = [vp, vp, vp, i64, vp]
        L.tdh_plan_execute_ragged.argtypes = [vp, vp, vp, vp, i64, vp]
        L.tdh_plan_query.argtypes = [vp, ctypes.POINTER(i64), ctypes.POINTER(i64)]
        L.tdh_plan_destroy.argtypes = [vp]
        L.tdh_last_error.argtypes = []
        L.tdh_last_error.restype = ctypes.c_char_p
        L.tdh_symbols.argtypes = [ctypes.c_int, i64, ctypes.POINTER(dbl), vp, vp, vp, vp, vp]
        L.tdh_pchol.argtypes = [vp, i64, i64, dbl, i64, vp, vp, ctypes.POINTER(i64), vp]
        L.tdh_pchol_noalloc.argtypes = [vp, i64, i64, dbl, i64, vp, vp, ctypes.POINTER(i64), vp]
        L.tdh_launch_count.argtypes = [ctypes.POINTER(i64)]
        L.tdh_alloc_stats.argtypes = [ctypes.POINTER(i64)]
        L.tdh_test_fail_alloc.argtypes = [i64]
        L.tdh_measure_fma_rate.argtypes = [ctypes.c_int, ctypes.POINTER(dbl), vp]
        L.tdh_plan_status.argtypes = [vp, ctypes.POINTER(ctypes.c_int), vp]
        L.tdh_test_tc_stall.argtypes = [ctypes.c_int]
        L.tdh_plan_execute_host.argtypes = [vp, vp, vp, i64, ctypes.c_int, vp]
        L.tdh_plan_execute_ragged_host.argtypes = [vp, vp, vp, vp, i64, vp]
        L.tdh_measure_dsmem_rate.argtypes = [ctypes.POINTER(dbl), vp]
        L.tdh_plan_schedule_count.argtypes = [vp, ctypes.POINTER(ctypes.c_int)]
        L.tdh_plan_schedule_info.argtypes = [vp, ctypes.c_int, ctypes.POINTER(ctypes.c_int)]
        L.tdh_plan_set_schedule.argtypes = [vp, ctypes.c_int, vp]
        L.tdh_plan_autotune.argtypes = [vp, i64, vp]
        L.tdh_schedules.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                    ctypes.POINTER(ctypes.c_int), ctypes.c_int,
                                    ctypes.POINTER(ctypes.c_int)]
        for name in EXPORTS:
            if name != "tdh_last_error":
                getattr(L, name).restype = ctypes.c_int
        _lib = L
    return _lib


def _check(rc):
    if rc != 0:
        raise TdhError(rc, lib().tdh_last_error().decode(errors="replace"))


def _torch():
    import torch
    return torch


def _stream(stream):
    torch = _torch()
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def _kind(kind):
    return KINDS[kind] if isinstance(kind, str) else int(kind)


class Plan:
    """A conversion plan (tdh_plan_create): symbols, pivoted Cholesky and FFT tables for
    vectors of n coefficients, built on the current CUDA device in float64.  tol is relative
    to max diag(H); with target=True it is the accuracy asked of the truncation instead
    (fewest rank terms whose residual bound gives max|beta_K - beta| <= tol ||alpha||_1).
    Without tol the plan is accuracy-targeted at half the precision's tolerance: 2.5e-6
    (float32), 5e-6 (split bfloat16, "bf16x3") or 5e-13 (float64)."""

    def __init__(self, kind, n, prec="fp32", tol=None, params=(), kmax=0, ragged=False,
                 target=None):
        self.kind = _kind(kind)
        self.prec = PRECS[prec] if isinstance(prec, str) else int(prec)
        if tol is None:
            # default: accuracy-targeted at half the precision's tolerance (5e-6 float32,
            # 1e-5 split bfloat16, 1e-12 float64, of ||alpha||_1), for every input
            tol = {FP64: 5e-13, FP32: 2.5e-6, BF16X3: 5e-6}.get(self.prec, 2.5e-6)
            target = True if target is None else target
        target = bool(target)
        p = _Params()
        for i, v in enumerate(params):
            p.p[i] = float(v)
        p.prec = self.prec
        p.flags = (FLAG_RAGGED if ragged else 0) | (FLAG_TARGET if target else 0)
        p.kmax = int(kmax)
        h = ctypes.c_void_p()
        _check(lib().tdh_plan_create(self.kind, int(n), ctypes.byref(p), float(tol),
                                     ctypes.byref(h)))
        self._h = h
        K, nn = ctypes.c_int64(), ctypes.c_int64()
        _check(lib().tdh_plan_query(h, ctypes.byref(K), ctypes.byref(nn)))
        self.K, self.n, self.tol = int(K.value), int(nn.value), float(tol)

    @property
    def dtype(self):
        torch = _torch()
        return torch.float64 if self.prec == FP64 else torch.float32

    def close(self):
        if getattr(self, "_h", None):
            lib().tdh_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _run(self, fn, x, out, stream, adjoint=0):
        torch = _torch()
        if x.dtype != self.dtype or x.shape[-1] != self.n or not x.is_contiguous():
            raise ValueError(f"expected a contiguous {self.dtype} tensor [..., {self.n}]")
        batch = x.numel() // self.n
        if x.device.type == "cpu":
            # host memory: the library pipelines the copies with the conversion
            res = out if out is not None else torch.empty(x.shape, dtype=x.dtype, pin_memory=True)
            if res.shape != x.shape or res.dtype != x.dtype or not res.is_contiguous():
                raise ValueError("out must be a contiguous host tensor like x")
            _check(lib().tdh_plan_execute_host(
                self._h, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(res.data_ptr()), batch,
                adjoint, _stream(stream)))
            return res
        od = out if out is not None else torch.empty_like(x)
        _check(fn(self._h, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(od.data_ptr()),
                  batch, _stream(stream)))
        return od

    def execute(self, x, out=None, stream=None):
        """beta = A alpha for every vector of x ([..., n], the plan's dtype).  A CUDA tensor
        runs on `stream` (default: torch's current stream) and returns asynchronously; a CPU
        tensor is copied in, converted and copied back (synchronise before reading)."""
        return self._run(lib().tdh_plan_execute, x, out, stream)

    def execute_ragged(self, x, offsets, out=None, stream=None):
        """Convert vectors of different lengths in one call: vector v is
        x[offsets[v]:offsets[v+1]] (offsets int64 with batch + 1 entries, every length <= n).
        CUDA tensors run on the device; a CPU x with CPU offsets is copied in, converted and
        copied back in overlapped chunks (synchronise before reading).  The plan must have
        been made with ragged=True."""
        torch = _torch()
        if x.dtype != self.dtype or not x.is_contiguous():
            raise ValueError(f"expected a contiguous {self.dtype} tensor")
        if x.device.type == "cpu":
            if offsets.dtype != torch.int64 or offsets.device.type != "cpu" or \
                    not offsets.is_contiguous():
                raise ValueError("host x needs contiguous host int64 offsets")
            res = out if out is not None else torch.empty(x.shape, dtype=x.dtype, pin_memory=True)
            if res.shape != x.shape or res.dtype != x.dtype or res.device.type != "cpu" or \
                    not res.is_contiguous():
                raise ValueError("out must be a contiguous host tensor like x")
            _check(lib().tdh_plan_execute_ragged_host(
                self._h, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(res.data_ptr()),
                ctypes.c_void_p(offsets.data_ptr()), offsets.numel() - 1, _stream(stream)))
            return res
        if x.device.type != "cuda":
            raise ValueError(f"expected a contiguous CUDA or host {self.dtype} tensor")
        if offsets.dtype != torch.int64 or offsets.device.type != "cuda":
            raise ValueError("offsets must be a CUDA int64 tensor")
        od = out if out is not None else torch.empty_like(x)
        _check(lib().tdh_plan_execute_ragged(
            self._h, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(od.data_ptr()),
            ctypes.c_void_p(offsets.data_ptr()), offsets.numel() - 1, _stream(stream)))
        return od

    def adjoint(self, g, out=None, stream=None):
        """A^T g for every vector of g (the transpose product)."""
        return self._run(lib().tdh_plan_execute_adjoint, g, out, stream, adjoint=1)

    STATUS = {1: "TIMEOUT", 2: "LENGTH", 4: "ALIAS", 8: "FAULT"}

    def status(self, stream=None):
        """TDH_STATUS_* bits the plan's kernels recorded since the last call, then cleared
        (tdh_plan_status; synchronises the stream): a set of names."""
        v = ctypes.c_int()
        _check(lib().tdh_plan_status(self._h, ctypes.byref(v), _stream(stream)))
        return {name for bit, name in self.STATUS.items() if v.value & bit}

    _SCHED_KEYS = ("logL", "logLC", "C", "R", "NT", "MINB", "index", "count")

    def schedules(self):
        """The execute schedule of each configuration (each T o H step, then each ragged
        length class): dicts with log2 L, log2 LC, cluster size C, radix R, threads NT,
        CTAs per SM MINB, and the schedule's index among `count` compiled ones."""
        n = ctypes.c_int()
        _check(lib().tdh_plan_schedule_count(self._h, ctypes.byref(n)))
        out = []
        for c in range(n.value):
            info = (ctypes.c_int * 8)()
            _check(lib().tdh_plan_schedule_info(self._h, c, info))
            out.append(dict(zip(self._SCHED_KEYS, list(info))))
        return out

    def set_schedule(self, index, stream=None):
        """Every configuration takes its schedule min(index, count - 1) (synchronous)."""
        _check(lib().tdh_plan_set_schedule(self._h, int(index), _stream(stream)))

    def autotune(self, batch, stream=None):
        """Time every compiled schedule on `batch` synthetic vectors and keep the fastest for
        each configuration (synchronous); returns schedules()."""
        _check(lib().tdh_plan_autotune(self._h, int(batch), _stream(stream)))
        return self.schedules()


def symbols(kind, n, params=(), stream=None):
    """Step a1 alone: (t, h, d1, d2) float64 CUDA tensors of the split A = D1 (T o H) D2."""
    torch = _torch()
    t = torch.empty(n, dtype=torch.float64, device="cuda")
    h = torch.empty(2 * n - 1, dtype=torch.float64, device="cuda")
    d1 = torch.empty(n, dtype=torch.float64, device="cuda")
    d2 = torch.empty(n, dtype=torch.float64, device="cuda")
    p = (ctypes.c_double * 4)(*([float(v) for v in params] + [0.0] * (4 - len(params))))
    ptr = lambda a: ctypes.c_void_p(a.data_ptr())
    _check(lib().tdh_symbols(_kind(kind), int(n), p, ptr(t), ptr(h), ptr(d1), ptr(d2),
                             _stream(stream)))
    return t, h, d1, d2


def pchol(h, n, j0, tol, kmax=128, stream=None):
    """Step a2 alone on a float64 CUDA Hankel generator h[2n-1]: returns (u [K][n], pivots)."""
    torch = _torch()
    kmax = int(min(kmax, n - j0))
    u = torch.zeros((kmax, n), dtype=torch.float64, device="cuda")
    piv = torch.zeros(kmax, dtype=torch.int64, device="cuda")
    K = ctypes.c_int64()
    _check(lib().tdh_pchol(ctypes.c_void_p(h.data_ptr()), int(n), int(j0), float(tol), kmax,
                           ctypes.c_void_p(u.data_ptr()), ctypes.c_void_p(piv.data_ptr()),
                           ctypes.byref(K), _stream(stream)))
    return u[: K.value].clone(), piv[: K.value].clone()


def compiled_schedules(prec, logL, ragged=False):
    """The compiled execute schedules for an FFT of 2^logL points (tdh_schedules, no device
    needed): dicts with log2 LC, C, R, NT, MINB and the multi-pass flag, default first."""
    prec = PRECS[prec] if isinstance(prec, str) else int(prec)
    n = ctypes.c_int()
    _check(lib().tdh_schedules(prec, int(logL), int(bool(ragged)), None, 0, ctypes.byref(n)))
    buf = (ctypes.c_int * (6 * max(n.value, 1)))()
    _check(lib().tdh_schedules(prec, int(logL), int(bool(ragged)), buf, n.value, ctypes.byref(n)))
    keys = ("logLC", "C", "R", "NT", "MINB", "multipass")
    return [dict(zip(keys, list(buf[6 * i:6 * i + 6]))) for i in range(n.value)]


def launch_count():
    """Kernel launches the library has enqueued for execute calls so far (tdh_launch_count)."""
    c = ctypes.c_int64()
    _check(lib().tdh_launch_count(ctypes.byref(c)))
    return int(c.value)


def alloc_stats():
    """(allocations made, plan blocks held, scratch blocks held) (tdh_alloc_stats)."""
    c = (ctypes.c_int64 * 3)()
    _check(lib().tdh_alloc_stats(c))
    return tuple(int(v) for v in c)


def inject_alloc_failure(k):
    """Make the k-th device allocation of the library from now on fail with NOMEM
    (tdh_test_fail_alloc; k = 0 cancels)."""
    _check(lib().tdh_test_fail_alloc(int(k)))


def measure_fma_rate(prec, stream=None):
    """FMA throughput of the current device in TFLOP/s (tdh_measure_fma_rate): prec "fp32"
    (FFMA) or "fp64" (DFMA), two flops per FMA."""
    prec = PRECS[prec] if isinstance(prec, str) else int(prec)
    v = ctypes.c_double()
    _check(lib().tdh_measure_fma_rate(prec, ctypes.byref(v), _stream(stream)))
    return float(v.value)


def measure_dsmem_rate(stream=None):
    """Distributed-shared-memory throughput in the cross stage's access pattern
    (tdh_measure_dsmem_rate): remote bytes per cycle per SM for loads, stores, and loads with
    stores (both directions counted) with every cluster resident, and loads with one cluster
    alone ("loads_one_cluster"), as a dict."""
    v = (ctypes.c_double * 4)()
    _check(lib().tdh_measure_dsmem_rate(v, _stream(stream)))
    return {"loads": float(v[0]), "stores": float(v[1]), "both": float(v[2]),
            "loads_one_cluster": float(v[3])}


def inject_tc_stall(on):
    """While on, split-bfloat16 executes issue no tensor-core products, so their bounded waits
    run out and TIMEOUT is recorded (tdh_test_tc_stall; outputs invalid)."""
    _check(lib().tdh_test_tc_stall(1 if on else 0))
