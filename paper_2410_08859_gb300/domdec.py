"""Python binding of the C ABI in ``include/domdec.h`` (argument marshalling only).

Every computation runs in ``_lib/libdomdec.so``; there is no fallback.  Arrays
may be NumPy float64 (host) or torch float64 tensors (host or CUDA); they must
be contiguous.  Functions keep the C names; ``DomDec`` is a small owning
wrapper around a handle.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

DOMDEC_OK, DOMDEC_WNOTCONV = 0, 1
DOMDEC_EINVAL, DOMDEC_ENOMEM, DOMDEC_ECUDA = -1, -2, -3
DOMDEC_ETOOBIG, DOMDEC_EARENA, DOMDEC_ESTATE, DOMDEC_ENOLIB = -4, -5, -6, -7
DOMDEC_EEMPTY, DOMDEC_ENONFINITE = -8, -9
STAGGERED, SWIFT, SAFE, GREEDY, LINE, STAGGERED_LINE = 0, 1, 2, 3, 4, 5
STRATEGIES = {"staggered": STAGGERED, "swift": SWIFT, "safe": SAFE, "greedy": GREEDY, "line": LINE,
              "staggered_line": STAGGERED_LINE}
FP32, FP64, MIXED = 0, 1, 2
SINKHORN_DENSE, SINKHORN_SEPARABLE, SINKHORN_TI = 0, 1, 4


class DomDecError(RuntimeError):
    def __init__(self, code, where):
        self.code = code
        super().__init__(f"{where}: {error_string(code)} ({code})")


class domdec_params(ctypes.Structure):
    _fields_ = [("eps", ctypes.c_double), ("lambda_", ctypes.c_double),
                ("basic_cell", ctypes.c_int), ("err", ctypes.c_double),
                ("trunc_thr", ctypes.c_double), ("tau", ctypes.c_double),
                ("strategy", ctypes.c_int), ("maxit", ctypes.c_int),
                ("newton_maxit", ctypes.c_int), ("precision", ctypes.c_int),
                ("box_margin", ctypes.c_int), ("max_ny", ctypes.c_int),
                ("arena_factor", ctypes.c_double), ("eps_init", ctypes.c_double),
                ("profile", ctypes.c_int), ("spill_slots", ctypes.c_int),
                ("cell_ctas", ctypes.c_int), ("cell_ti", ctypes.c_int), ("balance", ctypes.c_int),
                ("cell_split", ctypes.c_double)]


class domdec_stats(ctypes.Structure):
    _fields_ = [("sweeps", ctypes.c_longlong), ("cell_solves", ctypes.c_longlong),
                ("cell_iters", ctypes.c_longlong), ("maxit_cells", ctypes.c_longlong),
                ("greedy_steps", ctypes.c_longlong), ("safe_steps", ctypes.c_longlong),
                ("box_entries", ctypes.c_longlong), ("lse_terms", ctypes.c_longlong),
                ("box_points", ctypes.c_longlong), ("arena_regrows", ctypes.c_longlong),
                ("max_cell_iters", ctypes.c_int),
                ("max_ny", ctypes.c_int), ("cluster_regroups", ctypes.c_longlong)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


_LIB = None
_P = ctypes.c_void_p
_D = ctypes.c_double
_I = ctypes.c_int
_DP = ctypes.POINTER(ctypes.c_double)

_SIGS = {
    "domdec_default_params": (None, [ctypes.POINTER(domdec_params)]),
    "domdec_init": (_I, [ctypes.POINTER(_P), _P, _P, _I, ctypes.POINTER(domdec_params), _P, _P, _P]),
    "domdec_iterate": (_I, [_P, _I]),
    "domdec_autotune": (_I, [_P, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_double)]),
    "domdec_set_launch": (_I, [_P, ctypes.c_int, _D, ctypes.POINTER(ctypes.c_int)]),
    "domdec_reset": (_I, [_P, _P, _P, _P, _P, _D]),
    "domdec_set_eps": (_I, [_P, _D]),
    "domdec_set_tolerance": (_I, [_P, _D]),
    "domdec_sync": (_I, [_P]),
    "domdec_score": (_I, [_P, _DP]),
    "domdec_plan_marginals": (_I, [_P, _P, _P]),
    "domdec_duals": (_I, [_P, _P]),
    "domdec_pd_gap": (_I, [_P, _DP, _P]),
    "domdec_basic_costs": (_I, [_P, _P, _P]),
    "domdec_basic_marginals": (ctypes.c_longlong, [_P, ctypes.POINTER(ctypes.c_int), _P, ctypes.c_longlong]),
    "domdec_get_stats": (_I, [_P, ctypes.POINTER(domdec_stats)]),
    "domdec_decision_log": (_I, [_P, _DP, _I]),
    "domdec_kernel_times": (_I, [_P, _DP, ctypes.POINTER(ctypes.c_longlong), _I]),
    "domdec_cell_log": (_I, [_P, _DP, _I]),
    "domdec_free": (None, [_P]),
    "domdec_error_string": (ctypes.c_char_p, [_I]),
    "domdec_full_sinkhorn": (_I, [_P, _P, _I, _D, _D, _D, _I, _I, _I, _D, _I, _P, _P, _P, _DP, _P]),
    "domdec_full_sinkhorn_noalloc": (_I, [_P, _P, _I, _D, _D, _D, _I, _I, _I, _D, _I, _P, _P, _P, _DP, _P]),
    "domdec_uot_gradients": (_I, [_P, _P, _P, _P, _I, _D, _D, _I, _P, _P, _P, _DP, _P]),
    "domdec_gradients": (_I, [_P, _I, _P, _P, _P, _DP, _P]),
    "domdec_batch_create": (_I, [ctypes.POINTER(_P), ctypes.POINTER(_P), _I]),
    "domdec_batch_iterate": (_I, [_P, _I]),
    "domdec_batch_sync": (_I, [_P]),
    "domdec_batch_autotune": (_I, [_P, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_double)]),
    "domdec_batch_free": (None, [_P]),
    "domdec_probe_peaks": (_I, [_I, _DP, _P]),
    "domdec_probe_log": (_I, [_P, _P, _I, _P]),
}


def lib():
    """Load the in-tree library; raise if it has not been built."""
    global _LIB
    if _LIB is None:
        path = _build.LIB
        if not os.path.exists(path):
            raise RuntimeError(f"{path} is missing: build it first (python -c 'import __graft_entry__ as g; g.build()')")
        L = ctypes.CDLL(path)
        for name, (res, args) in _SIGS.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _LIB = L
    return _LIB


def error_string(code):
    try:
        return lib().domdec_error_string(int(code)).decode()
    except Exception:  # library unavailable while formatting an error
        return f"error {code}"


def _check(rc, where):
    if rc < 0:
        raise DomDecError(rc, where)
    return rc


def _ptr(a, n=None, writable=False):
    """Raw pointer of a contiguous float64 NumPy array or torch tensor (or None)."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        if a.dtype != np.float64 or not a.flags["C_CONTIGUOUS"]:
            raise TypeError("expected a C-contiguous float64 array")
        if writable and not a.flags["WRITEABLE"]:
            raise TypeError("array is read-only")
        if n is not None and a.size != n:
            raise ValueError(f"expected {n} elements, got {a.size}")
        return a.ctypes.data
    import torch  # torch tensors: device memory owned by PyTorch
    if isinstance(a, torch.Tensor):
        if a.dtype != torch.float64 or not a.is_contiguous():
            raise TypeError("expected a contiguous float64 tensor")
        if n is not None and a.numel() != n:
            raise ValueError(f"expected {n} elements, got {a.numel()}")
        return a.data_ptr()
    raise TypeError(f"unsupported array type {type(a)}")


def _stream_ptr(stream):
    if stream is None:
        try:
            import torch
            if torch.cuda.is_available():
                return torch.cuda.current_stream().cuda_stream
        except Exception:
            pass
        return None
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def domdec_default_params(**kw):
    p = domdec_params()
    lib().domdec_default_params(ctypes.byref(p))
    for k, v in kw.items():
        if k in ("lam", "lambda"):
            k = "lambda_"
        if k == "strategy" and isinstance(v, str):
            v = STRATEGIES[v]
        if k == "precision" and isinstance(v, str):
            v = {"fp32": FP32, "fp64": FP64}[v]
        setattr(p, k, v)
    return p


def domdec_init(mu, nu, N, params, alpha0=None, beta0=None, stream=None):
    h = _P()
    n = N * N
    rc = lib().domdec_init(ctypes.byref(h), _ptr(mu, n), _ptr(nu, n), int(N), ctypes.byref(params),
                           _ptr(alpha0, n), _ptr(beta0, n), _stream_ptr(stream))
    _check(rc, "domdec_init")
    return h


def domdec_reset(h, mu, nu, N, alpha0=None, beta0=None, eps_init=0.0):
    n = N * N
    return _check(lib().domdec_reset(h, _ptr(mu, n), _ptr(nu, n), _ptr(alpha0, n), _ptr(beta0, n),
                                     float(eps_init)), "domdec_reset")


def domdec_iterate(h, n_sweeps):
    return _check(lib().domdec_iterate(h, int(n_sweeps)), "domdec_iterate")


def domdec_set_eps(h, eps):
    return _check(lib().domdec_set_eps(h, float(eps)), "domdec_set_eps")


def domdec_set_tolerance(h, err):
    _check(lib().domdec_set_tolerance(h, float(err)), "domdec_set_tolerance")


def domdec_sync(h):
    return _check(lib().domdec_sync(h), "domdec_sync")


def domdec_score(h):
    out = (ctypes.c_double * 6)()
    _check(lib().domdec_score(h, out), "domdec_score")
    return np.array(out[:])


def domdec_plan_marginals(h, PX, PY):
    return _check(lib().domdec_plan_marginals(h, _ptr(PX, writable=True), _ptr(PY, writable=True)),
                  "domdec_plan_marginals")


def domdec_duals(h, alpha):
    return _check(lib().domdec_duals(h, _ptr(alpha, writable=True)), "domdec_duals")


def domdec_basic_costs(h, nbasic):
    """(C, H): the tracked transport cost and entropy of every basic cell's plan part."""
    C, H = np.empty(nbasic), np.empty(nbasic)
    _check(lib().domdec_basic_costs(h, C.ctypes.data, H.ctypes.data), "domdec_basic_costs")
    return C, H


def domdec_pd_gap(h, beta=None):
    out = (ctypes.c_double * 5)()
    _check(lib().domdec_pd_gap(h, out, _ptr(beta, writable=True)), "domdec_pd_gap")
    return np.array(out[:])


def domdec_basic_marginals(h, nbasic):
    box = (ctypes.c_int * (4 * nbasic))()
    total = _check(lib().domdec_basic_marginals(h, box, None, 0), "domdec_basic_marginals")
    vals = np.empty(max(total, 1))
    _check(lib().domdec_basic_marginals(h, box, vals.ctypes.data, total), "domdec_basic_marginals")
    return np.array(box[:], dtype=np.int64).reshape(nbasic, 4), vals[:total]


def domdec_decision_log(h, max_records=4096):
    """(n, 4) array of (E_hat, E(1), E(safe), theta) per sub-batch, oldest first."""
    out = (ctypes.c_double * (4 * max_records))()
    cnt = _check(lib().domdec_decision_log(h, out, int(max_records)), "domdec_decision_log")
    return np.array(out[:4 * cnt]).reshape(cnt, 4)


def domdec_kernel_times(h, reset=True):
    """(ms[4], launches[4]) per kernel class: cell solve, decision, apply, compaction."""
    ms = (ctypes.c_double * 4)()
    n = (ctypes.c_longlong * 4)()
    _check(lib().domdec_kernel_times(h, ms, n, int(reset)), "domdec_kernel_times")
    return np.array(ms[:]), np.array(n[:])


def domdec_cell_log(h, max_records=4096):
    """(n, 9) array per cell of the last sub-batch: k0, l0, H, W, iters, status, gap, spill slot,
    solve duration (us)."""
    out = (ctypes.c_double * (9 * max_records))()
    cnt = _check(lib().domdec_cell_log(h, out, int(max_records)), "domdec_cell_log")
    return np.array(out[:9 * cnt]).reshape(cnt, 9)


def domdec_get_stats(h):
    s = domdec_stats()
    _check(lib().domdec_get_stats(h, ctypes.byref(s)), "domdec_get_stats")
    return s.as_dict()


def domdec_free(h):
    if h:
        lib().domdec_free(h)


def domdec_full_sinkhorn(mu, nu, N, eps, lam, eps_start=None, variant=SINKHORN_SEPARABLE,
                         precision=FP64, maxit=10000, err=2e-5, check_every=10, beta_in=None,
                         alpha=None, beta=None, stream=None):
    """Global unbalanced Sinkhorn; returns (iterations, PD/lam, primal, dual, rc)."""
    out = (ctypes.c_double * 4)()
    n = N * N
    rc = lib().domdec_full_sinkhorn(_ptr(mu, n), _ptr(nu, n), int(N),
                                    float(eps if eps_start is None else eps_start), float(eps), float(lam),
                                    int(variant), int(precision), int(maxit), float(err), int(check_every),
                                    _ptr(beta_in, n), _ptr(alpha, n, True), _ptr(beta, n, True), out,
                                    _stream_ptr(stream))
    _check(rc, "domdec_full_sinkhorn")
    return int(out[0]), out[1], out[2], out[3], rc


def domdec_full_sinkhorn_noalloc(mu, nu, N, eps, lam, alpha, beta, eps_start=None,
                                 variant=SINKHORN_SEPARABLE, precision=FP64, maxit=10000, err=2e-5,
                                 check_every=10, beta_in=None, stream=None):
    """Allocation-free global Sinkhorn: device tensors only, N <= 256 (see
    include/domdec.h).  Returns (iterations, PD/lam, primal, dual, rc).
    NumPy arrays and tensors that do not live on the current CUDA device are
    rejected here, before the library is called (the C entry point rejects
    them too)."""
    import torch
    for name, a in (("mu", mu), ("nu", nu), ("alpha", alpha), ("beta", beta), ("beta_in", beta_in)):
        if a is None and name == "beta_in":
            continue
        if not (isinstance(a, torch.Tensor) and a.is_cuda and a.device.index == torch.cuda.current_device()):
            raise TypeError(f"domdec_full_sinkhorn_noalloc: {name} must be a tensor on the current CUDA device")
    out = (ctypes.c_double * 4)()
    n = N * N
    rc = lib().domdec_full_sinkhorn_noalloc(_ptr(mu, n), _ptr(nu, n), int(N),
                                            float(eps if eps_start is None else eps_start), float(eps),
                                            float(lam), int(variant), int(precision), int(maxit), float(err),
                                            int(check_every), _ptr(beta_in, n), _ptr(alpha, n, True),
                                            _ptr(beta, n, True), out, _stream_ptr(stream))
    _check(rc, "domdec_full_sinkhorn_noalloc")
    return int(out[0]), out[1], out[2], out[3], rc


def domdec_uot_gradients(mu, nu, alpha, beta, N, eps, lam, precision=FP64, grad_mu=None, grad_nu=None,
                         grad_x=None, stream=None):
    """Envelope-theorem gradients of the UOT value at potentials (alpha, beta)
    into grad_mu, grad_nu (N*N) and grad_x (2*N*N); returns
    [D(alpha, beta), |mu|, |nu|, |P_X pi|, |P_Y pi|]."""
    out = (ctypes.c_double * 5)()
    n = N * N
    rc = lib().domdec_uot_gradients(_ptr(mu, n), _ptr(nu, n), _ptr(alpha, n), _ptr(beta, n), int(N), float(eps),
                                    float(lam), int(precision), _ptr(grad_mu, n, True), _ptr(grad_nu, n, True),
                                    _ptr(grad_x, 2 * n, True), out, _stream_ptr(stream))
    _check(rc, "domdec_uot_gradients")
    return list(out)


def domdec_gradients(h, N, precision=FP64, grad_mu=None, grad_nu=None, grad_x=None, beta=None):
    """domdec_uot_gradients at a handle's state (alpha stitched, beta_star)."""
    out = (ctypes.c_double * 5)()
    n = N * N
    _check(lib().domdec_gradients(h, int(precision), _ptr(grad_mu, n, True), _ptr(grad_nu, n, True),
                                  _ptr(grad_x, 2 * n, True), out, _ptr(beta, n, True)), "domdec_gradients")
    return list(out)


def domdec_probe_peaks(iters=20000, stream=None):
    """MUFU ex2 and FFMA throughput of the current device: dict with ex2/s,
    ex2 per SM per clock, FFMA/s, FFMA per SM per clock, SM clocks, SM count."""
    out = (ctypes.c_double * 8)()
    _check(lib().domdec_probe_peaks(int(iters), out, _stream_ptr(stream)), "domdec_probe_peaks")
    return {"ex2_per_s": out[0], "ex2_per_sm_clk": out[1], "ex2_sm_mhz": out[2],
            "ffma_per_s": out[3], "ffma_per_sm_clk": out[4], "ffma_sm_mhz": out[5],
            "sms": int(out[6]), "blocks": int(out[7])}


def domdec_probe_log(x, y, stream=None):
    """y = the library's double logarithm of x (device float64 tensors)."""
    _check(lib().domdec_probe_log(_ptr(x), _ptr(y, writable=True), int(x.numel()), _stream_ptr(stream)),
           "domdec_probe_log")


class DomDecBatch:
    """Many independent DomDec problems swept together (the handles stay
    owned by their DomDec objects, which must outlive the batch)."""

    def __init__(self, problems):
        self.problems = list(problems)
        arr = (_P * len(self.problems))(*[p.h for p in self.problems])
        b = _P()
        _check(lib().domdec_batch_create(ctypes.byref(b), arr, len(self.problems)), "domdec_batch_create")
        self.b = b

    def iterate(self, n=1):
        _check(lib().domdec_batch_iterate(self.b, int(n)), "domdec_batch_iterate")
        return self

    def sync(self):
        return _check(lib().domdec_batch_sync(self.b), "domdec_batch_sync")

    def autotune(self):
        """Time the candidate cluster sizes / split thresholds for one sweep each
        and keep the fastest; returns (cluster CTAs, split factor)."""
        c = ctypes.c_int(0)
        f = ctypes.c_double(0.0)
        _check(lib().domdec_batch_autotune(self.b, ctypes.byref(c), ctypes.byref(f)), "domdec_batch_autotune")
        return c.value, f.value

    def close(self):
        if self.b:
            lib().domdec_batch_free(self.b)
            self.b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class DomDec:
    """Owning wrapper: ``DomDec(mu, nu, eps=..., lam=..., s=...)``."""

    def __init__(self, mu, nu, eps, lam, s, alpha0=None, beta0=None, stream=None, **params):
        mu_a = mu if not isinstance(mu, np.ndarray) else np.ascontiguousarray(mu, dtype=np.float64).ravel()
        nu_a = nu if not isinstance(nu, np.ndarray) else np.ascontiguousarray(nu, dtype=np.float64).ravel()
        n = mu_a.size if isinstance(mu_a, np.ndarray) else mu_a.numel()
        self.N = int(round(n ** 0.5))
        self.s = s
        self.nbasic = (self.N // s) ** 2
        self.params = domdec_default_params(eps=eps, lam=lam, basic_cell=s, **params)
        a0 = None if alpha0 is None else np.ascontiguousarray(alpha0, dtype=np.float64).ravel() \
            if isinstance(alpha0, np.ndarray) else alpha0
        b0 = None if beta0 is None else np.ascontiguousarray(beta0, dtype=np.float64).ravel() \
            if isinstance(beta0, np.ndarray) else beta0
        self.h = domdec_init(mu_a, nu_a, self.N, self.params, a0, b0, stream)

    def iterate(self, n=1):
        domdec_iterate(self.h, n)
        return self

    def autotune(self):
        """Time the cell-launch candidates (cluster size, split threshold) for one
        sweep each and keep the fastest; returns (cluster CTAs, split factor)."""
        c = ctypes.c_int(0)
        f = ctypes.c_double(0.0)
        _check(lib().domdec_autotune(self.h, ctypes.byref(c), ctypes.byref(f)), "domdec_autotune")
        return c.value, f.value

    def set_launch(self, cluster_ctas, split):
        """Set the cell launch shape (domdec_set_launch); returns the cluster size in use."""
        c = ctypes.c_int(0)
        _check(lib().domdec_set_launch(self.h, int(cluster_ctas), float(split), ctypes.byref(c)),
               "domdec_set_launch")
        return c.value

    def reset(self, mu, nu, alpha0=None, beta0=None, eps_init=0.0):
        """Load a new problem of the same size into this handle (domdec_reset)."""
        domdec_reset(self.h, mu, nu, self.N, alpha0, beta0, eps_init)
        return self

    def sync(self):
        return domdec_sync(self.h)

    def set_eps(self, eps):
        domdec_set_eps(self.h, eps)

    def set_tolerance(self, err):
        domdec_set_tolerance(self.h, err)

    def score(self):
        return domdec_score(self.h)

    def marginals(self):
        n = self.N * self.N
        PX, PY = np.empty(n), np.empty(n)
        domdec_plan_marginals(self.h, PX, PY)
        return PX, PY

    def duals(self):
        a = np.empty(self.N * self.N)
        domdec_duals(self.h, a)
        return a

    def pd_gap(self, with_beta=False):
        beta = np.empty(self.N * self.N) if with_beta else None
        out = domdec_pd_gap(self.h, beta)
        return (out, beta) if with_beta else out

    def basic_marginals(self):
        return domdec_basic_marginals(self.h, self.nbasic)

    def basic_costs(self):
        return domdec_basic_costs(self.h, self.nbasic)

    def gradients(self, precision=FP64, grad_mu=None, grad_nu=None, grad_x=None, beta=None):
        """d(score)/d mu, d(score)/d nu, d(score)/d x at the current state
        (NumPy arrays unless buffers are given); returns (g_mu, g_nu, g_x, out)."""
        n = self.N * self.N
        g_mu = np.empty(n) if grad_mu is None else grad_mu
        g_nu = np.empty(n) if grad_nu is None else grad_nu
        g_x = np.empty(2 * n) if grad_x is None else grad_x
        out = domdec_gradients(self.h, self.N, precision, g_mu, g_nu, g_x, beta)
        return g_mu, g_nu, g_x, out

    def stats(self):
        return domdec_get_stats(self.h)

    def kernel_times(self, reset=True):
        return domdec_kernel_times(self.h, reset)

    def cell_log(self, max_records=4096):
        return domdec_cell_log(self.h, max_records)

    def decisions(self, max_records=4096):
        return domdec_decision_log(self.h, max_records)

    def close(self):
        if self.h:
            domdec_free(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
