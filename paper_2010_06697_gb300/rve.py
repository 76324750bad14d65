"""ctypes binding of the C ABI in include/rve.h (same names, argument marshalling only).

Every step of the ADMM iteration runs in ``lib/librve.so``; this module only
converts numpy / torch arguments to pointers and status codes to exceptions.
It raises ImportError-like RuntimeError when the library has not been built:
there is no fallback path.

``Rve`` is a small owner object around one handle.  By default it takes its
device workspace from a torch CUDA tensor (``rve_create_in``), so PyTorch's
caching allocator provides the memory; pass ``use_torch=False`` to let the
library call cudaMalloc itself (``rve_create``).
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "lib", "librve.so")

RVE_OK = 0
RVE_E_INVALID_ARG = -1
RVE_E_OOM = -2
RVE_E_NOT_CONVERGED = -3
RVE_E_NUMERICAL = -4
RVE_E_CUDA = -5
RVE_E_BUSY = -6
RVE_E_STATE = -7
RVE_E_NOT_FOUND = -8

RVE_NEOHOOKE, RVE_LINEAR, RVE_LCE = 0, 1, 2
RVE_FP64, RVE_MIXED, RVE_FP32 = 0, 1, 2
RVE_RHO_FIXED, RVE_RHO_ADAPTIVE = 0, 1
RVE_LAMBDA0_STRESS, RVE_LAMBDA0_ZERO = 0, 1
RVE_FIELD_F, RVE_FIELD_LAMBDA, RVE_FIELD_U, RVE_FIELD_N = 0, 1, 2, 3

MODELS = {"neohookean": RVE_NEOHOOKE, "linear": RVE_LINEAR, "lce": RVE_LCE}
PRECISIONS = {"fp64": RVE_FP64, "mixed": RVE_MIXED, "fp32": RVE_FP32}


class rve_options(ctypes.Structure):
    _fields_ = [
        ("precision", ctypes.c_int),
        ("rho_policy", ctypes.c_int),
        ("lambda0", ctypes.c_int),
        ("max_iter", ctypes.c_int),
        ("newton_max", ctypes.c_int),
        ("newton_tol", ctypes.c_double),
        ("rho_kappa", ctypes.c_double),
        ("rho_tau", ctypes.c_double),
        ("rho_min", ctypes.c_double),
        ("mu_ref", ctypes.c_double),
        ("mixed_switch", ctypes.c_double),
        ("check_every", ctypes.c_int),
        ("use_graph", ctypes.c_int),
        ("local_ratio", ctypes.c_double),
        ("local_fraction", ctypes.c_double),
    ]


class rve_solve_info(ctypes.Structure):
    _fields_ = [
        ("iterations", ctypes.c_int),
        ("fp64_iterations", ctypes.c_int),
        ("converged", ctypes.c_int),
        ("status", ctypes.c_int),
        ("r_p", ctypes.c_double),
        ("r_d", ctypes.c_double),
        ("rho", ctypes.c_double),
        ("mu_ref", ctypes.c_double),
        ("newton_max_iters", ctypes.c_int),
        ("newton_fail", ctypes.c_longlong),
        ("time_ms", ctypes.c_double),
        ("launches", ctypes.c_longlong),
        ("r_l", ctypes.c_double),
    ]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class rve_bloch_info(ctypes.Structure):
    _fields_ = [
        ("iterations", ctypes.c_int),
        ("converged", ctypes.c_int),
        ("beta", ctypes.c_double),
        ("rayleigh", ctypes.c_double),
        ("r_p", ctypes.c_double),
        ("r_d", ctypes.c_double),
        ("time_ms", ctypes.c_double),
        ("launches", ctypes.c_longlong),
        ("fail", ctypes.c_int),
        ("rho", ctypes.c_double),
        ("float_iterations", ctypes.c_int),
    ]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


_VP = ctypes.c_void_p
_I = ctypes.c_int
_D = ctypes.c_double
_SZ = ctypes.c_size_t
_PD = ctypes.POINTER(ctypes.c_double)

SIGNATURES = {
    "rve_default_options": (None, [ctypes.POINTER(rve_options)]),
    "rve_workspace_bytes": (_SZ, [_I, _I, _I, ctypes.POINTER(rve_options)]),
    "rve_create": (_I, [ctypes.POINTER(_VP), _I, _I, _I, ctypes.POINTER(rve_options), _VP]),
    "rve_create_in": (_I, [ctypes.POINTER(_VP), _I, _I, _I, ctypes.POINTER(rve_options), _VP, _VP, _SZ]),
    "rve_destroy": (None, [_VP]),
    "rve_set_material": (_I, [_VP, ctypes.POINTER(ctypes.c_uint8), _I, _PD, _I, _PD]),
    "rve_solve": (_I, [_VP, _PD, _D, _D, ctypes.POINTER(rve_solve_info)]),
    "rve_stress": (_I, [_VP, _PD]),
    "rve_mean_lambda": (_I, [_VP, _PD]),
    "rve_get_field": (_I, [_VP, _I, _PD]),
    "rve_set_field": (_I, [_VP, _I, _PD]),
    "rve_reset": (_I, [_VP]),
    "rve_history": (_I, [_VP, _PD, _PD, _PD, _I]),
    "rve_history_local": (_I, [_VP, _PD, _I]),
    "rve_solve_mixed": (_I, [_VP, _PD, ctypes.c_uint, _D, _D, ctypes.POINTER(rve_solve_info)]),
    "rve_macro_gradient": (_I, [_VP, _PD]),
    "rve_solve_path": (_I, [_VP, _PD, _I, ctypes.c_uint, _D, _D, _PD, _PD, ctypes.POINTER(rve_solve_info)]),
    "rve_bloch": (_I, [_VP, ctypes.POINTER(_I), _PD, _D, _D, _I, _PD, _PD, ctypes.POINTER(rve_bloch_info)]),
    "rve_strerror": (ctypes.c_char_p, [_I]),
    "rve_set_profiling": (_I, [_VP, _I]),
    "rve_stress_noalloc": (_I, [_I, _I, _I, _VP, _VP, _VP, _I, _I, _VP, _VP]),
    "rve_batch_create": (_I, [ctypes.POINTER(_VP), ctypes.POINTER(_VP), _I, _VP]),
    "rve_batch_solve": (_I, [_VP, _PD, _PD, _D, ctypes.POINTER(rve_solve_info)]),
    "rve_batch_destroy": (None, [_VP]),
    "rve_server_create": (_I, [ctypes.POINTER(_VP), _SZ, ctypes.POINTER(rve_options), _VP]),
    "rve_server_submit": (_I, [_VP, _I, _I, _I, ctypes.POINTER(ctypes.c_uint8), _I, _PD, _I, _PD, _PD, _D, _D,
                               ctypes.POINTER(ctypes.c_longlong)]),
    "rve_server_step": (_I, [_VP, ctypes.POINTER(_I), ctypes.POINTER(_I)]),
    "rve_server_poll": (_I, [_VP, ctypes.c_longlong, _PD, ctypes.POINTER(rve_solve_info), _PD, _PD]),
    "rve_server_cancel": (_I, [_VP, ctypes.c_longlong]),
    "rve_server_stats": (_I, [_VP, ctypes.POINTER(ctypes.c_longlong), ctypes.POINTER(ctypes.c_longlong),
                              ctypes.POINTER(ctypes.c_longlong), ctypes.POINTER(_SZ)]),
    "rve_server_destroy": (None, [_VP]),
    "rve_autotune": (_I, [_I, _I, _I, ctypes.c_char_p, _PD]),
    "rve_autotune_load": (_I, [ctypes.c_char_p]),
    "rve_kernel_times": (_I, [_VP, _I, _PD, ctypes.POINTER(ctypes.c_longlong), _I]),
}

KCLASS_NAMES = ["local", "local_first", "xfwd", "fwd_y", "solve", "inv_y", "xinv", "local_r", "xfwd_incr",
                "xinv_incr"]

_lib = None


def lib():
    """Load librve.so (once).  Raises RuntimeError if it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with __graft_entry__.build()")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


class RveError(RuntimeError):
    def __init__(self, code, where=""):
        self.code = code
        msg = lib().rve_strerror(code).decode()
        super().__init__(f"{where}: {msg} ({code})" if where else f"{msg} ({code})")


def _check(code, where):
    if code != RVE_OK:
        raise RveError(code, where)
    return code


def _dptr(a):
    return a.ctypes.data_as(_PD)


# ------------------------------------------------------------------ ABI-named thin wrappers

def rve_default_options():
    o = rve_options()
    lib().rve_default_options(ctypes.byref(o))
    return o


def rve_workspace_bytes(dim, n, model, opt=None):
    return int(lib().rve_workspace_bytes(dim, n, model, ctypes.byref(opt) if opt is not None else None))


def rve_strerror(code):
    return lib().rve_strerror(code).decode()


def rve_create(dim, n, model, opt=None, stream=None):
    h = _VP()
    rc = lib().rve_create(ctypes.byref(h), dim, n, model, ctypes.byref(opt) if opt is not None else None,
                          _VP(stream or 0))
    return rc, h


def rve_create_in(dim, n, model, opt, stream, workspace_ptr, nbytes):
    h = _VP()
    rc = lib().rve_create_in(ctypes.byref(h), dim, n, model, ctypes.byref(opt) if opt is not None else None,
                             _VP(stream or 0), _VP(workspace_ptr), nbytes)
    return rc, h


def rve_destroy(h):
    lib().rve_destroy(h)


def rve_set_material(h, phase, params, n0=None):
    ph = np.ascontiguousarray(phase, dtype=np.uint8)
    par = np.ascontiguousarray(params, dtype=np.float64)
    nphase, nparam = par.shape
    n0p = None
    if n0 is not None:
        n0a = np.ascontiguousarray(n0, dtype=np.float64)
        n0p = _dptr(n0a)
    return lib().rve_set_material(h, ph.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8)), nphase, _dptr(par),
                                  nparam, n0p)


def rve_solve(h, Fbar, rho, tol):
    fb = np.ascontiguousarray(np.asarray(Fbar, dtype=np.float64).reshape(3, 3))
    info = rve_solve_info()
    rc = lib().rve_solve(h, _dptr(fb), float(rho), float(tol), ctypes.byref(info))
    return rc, info


def free_mask_bits(free):
    """(3, 3) boolean array of free <F> components -> the bit mask of rve_solve_mixed."""
    f = np.asarray(free, dtype=bool).reshape(3, 3)
    return int(sum(1 << (3 * i + j) for i in range(3) for j in range(3) if f[i, j]))


def rve_solve_mixed(h, Fbar, free, rho, tol):
    fb = np.ascontiguousarray(np.asarray(Fbar, dtype=np.float64).reshape(3, 3))
    info = rve_solve_info()
    rc = lib().rve_solve_mixed(h, _dptr(fb), free_mask_bits(free), float(rho), float(tol), ctypes.byref(info))
    return rc, info


def rve_macro_gradient(h):
    F = np.zeros(9)
    rc = lib().rve_macro_gradient(h, _dptr(F))
    return rc, F.reshape(3, 3)


def rve_stress(h):
    S = np.zeros(9)
    rc = lib().rve_stress(h, _dptr(S))
    return rc, S.reshape(3, 3)


def rve_mean_lambda(h):
    S = np.zeros(9)
    rc = lib().rve_mean_lambda(h, _dptr(S))
    return rc, S.reshape(3, 3)


def rve_get_field(h, which, out):
    return lib().rve_get_field(h, which, _dptr(out))


def rve_set_field(h, which, arr):
    a = np.ascontiguousarray(arr, dtype=np.float64)
    return lib().rve_set_field(h, which, _dptr(a))


def rve_reset(h):
    return lib().rve_reset(h)


def rve_history(h, cap):
    rp, rd, rho = np.zeros(cap), np.zeros(cap), np.zeros(cap)
    cnt = lib().rve_history(h, _dptr(rp), _dptr(rd), _dptr(rho), cap)
    if cnt < 0:
        return cnt, None
    return cnt, np.stack([rp[:cnt], rd[:cnt], rho[:cnt]], axis=1)


def rve_history_local(h, cap):
    rl = np.zeros(cap)
    cnt = lib().rve_history_local(h, _dptr(rl), cap)
    if cnt < 0:
        return cnt, None
    return cnt, rl[:cnt]


def rve_bloch(h, k, p0, rho, tol, max_iter, want_p=True):
    """Modulus of stability beta_k (see include/rve.h).  k: d non-zero ints; p0: complex
    (d, *grid).  Returns (rc, info, p or None, history (iterations, 4): r_p, r_d, sigma, rho)."""
    kk = (ctypes.c_int * 3)(*(list(int(x) for x in k) + [1] * (3 - len(k))))
    p = np.ascontiguousarray(np.asarray(p0, dtype=np.complex128))
    out = np.zeros_like(p) if want_p else None
    hist = np.zeros(4 * int(max_iter))
    info = rve_bloch_info()
    rc = lib().rve_bloch(h, kk, p.view(np.float64).ctypes.data_as(_PD), float(rho), float(tol), int(max_iter),
                         out.view(np.float64).ctypes.data_as(_PD) if want_p else None, _dptr(hist),
                         ctypes.byref(info))
    return rc, info, out, hist.reshape(-1, 4)[: info.iterations]


def rve_stress_noalloc(dim, n, model, F_ptr, phase_ptr, params_ptr, nphase, nparam, S_ptr, stream=None):
    """Device pointers in, device pointer out; see include/rve.h (no device allocation)."""
    return lib().rve_stress_noalloc(dim, n, model, _VP(F_ptr), _VP(phase_ptr), _VP(params_ptr), nphase, nparam,
                                    _VP(S_ptr), _VP(stream or 0))


def rve_autotune(dim, n, precision="mixed", cache_path=None):
    """Tune the FFT geometry of N^d grids; returns the tuned FFT milliseconds per iteration."""
    p = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
    ms = ctypes.c_double()
    rc = lib().rve_autotune(dim, n, p, cache_path.encode() if cache_path else None, ctypes.byref(ms))
    _check(rc, "rve_autotune")
    return ms.value


def rve_autotune_load(cache_path):
    return lib().rve_autotune_load(cache_path.encode())


def rve_set_profiling(h, on):
    return lib().rve_set_profiling(h, 1 if on else 0)


def rve_kernel_times(h, fp64):
    ms = np.zeros(len(KCLASS_NAMES))
    n = np.zeros(len(KCLASS_NAMES), dtype=np.int64)
    rc = lib().rve_kernel_times(h, 1 if fp64 else 0, _dptr(ms), n.ctypes.data_as(ctypes.POINTER(ctypes.c_longlong)),
                                len(KCLASS_NAMES))
    return rc, ms, n


def rve_batch_create(handles, stream=None):
    arr = (_VP * len(handles))(*[h.value if isinstance(h, _VP) else h for h in handles])
    b = _VP()
    rc = lib().rve_batch_create(ctypes.byref(b), arr, len(handles), _VP(stream or 0))
    return rc, b


def rve_batch_solve(b, Fbars, rhos, tol):
    fb = np.ascontiguousarray(np.asarray(Fbars, dtype=np.float64).reshape(-1, 9))
    rh = np.ascontiguousarray(np.asarray(rhos, dtype=np.float64).reshape(-1))
    infos = (rve_solve_info * fb.shape[0])()
    rc = lib().rve_batch_solve(b, _dptr(fb), _dptr(rh), float(tol), infos)
    return rc, list(infos)


def rve_batch_destroy(b):
    lib().rve_batch_destroy(b)


class Batch:
    """Batched solves over existing Rve objects (kept alive by this object)."""

    def __init__(self, members, stream=None):
        self.members = list(members)
        if stream is None:
            import torch
            stream = torch.cuda.current_stream().cuda_stream
        rc, b = rve_batch_create([m.h for m in self.members], stream)
        _check(rc, "rve_batch_create")
        self.b = b

    def solve(self, Fbars, rhos, tol):
        rc, infos = rve_batch_solve(self.b, Fbars, rhos, tol)
        if rc not in (RVE_OK, RVE_E_NOT_CONVERGED):
            raise RveError(rc, "rve_batch_solve")
        return infos

    def close(self):
        if self.b is not None:
            rve_batch_destroy(self.b)
            self.b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """Continuous-batching server (rve_server_*): submit requests, step, poll results."""

    def __init__(self, mem_budget_bytes, precision="mixed", stream=None, **options):
        opt = rve_default_options()
        opt.precision = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
        for k, v in options.items():
            setattr(opt, k, v)
        self.opt = opt
        if stream is None:
            import torch
            stream = torch.cuda.current_stream().cuda_stream
        h = _VP()
        _check(lib().rve_server_create(ctypes.byref(h), int(mem_budget_bytes), ctypes.byref(opt), _VP(stream or 0)),
               "rve_server_create")
        self.s = h

    def submit(self, phase, params, Fbar, rho, tol, model="neohookean", n0=None):
        ph = np.ascontiguousarray(phase, dtype=np.uint8)
        par = np.ascontiguousarray(params, dtype=np.float64)
        fb = np.ascontiguousarray(np.asarray(Fbar, dtype=np.float64).reshape(3, 3))
        n0p = None
        if n0 is not None:
            n0a = np.ascontiguousarray(n0, dtype=np.float64)
            n0p = _dptr(n0a)
        t = ctypes.c_longlong()
        m = MODELS[model] if isinstance(model, str) else int(model)
        rc = lib().rve_server_submit(self.s, ph.ndim, ph.shape[0], m, ph.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8)),
                                     par.shape[0], _dptr(par), par.shape[1], n0p, _dptr(fb), float(rho), float(tol),
                                     ctypes.byref(t))
        _check(rc, "rve_server_submit")
        return t.value

    def step(self):
        a, q = _I(), _I()
        _check(lib().rve_server_step(self.s, ctypes.byref(a), ctypes.byref(q)), "rve_server_step")
        return a.value, q.value

    def poll(self, ticket):
        """None while pending; else (status, S 3x3, info, latency_ms, queue_ms)."""
        S = np.zeros(9)
        info = rve_solve_info()
        lat, qw = ctypes.c_double(), ctypes.c_double()
        rc = lib().rve_server_poll(self.s, ticket, _dptr(S), ctypes.byref(info), ctypes.byref(lat), ctypes.byref(qw))
        if rc == RVE_E_BUSY:
            return None
        if rc == RVE_E_NOT_FOUND or rc in (RVE_E_INVALID_ARG, RVE_E_CUDA):
            raise RveError(rc, "rve_server_poll")
        return rc, S.reshape(3, 3), info, lat.value, qw.value

    def cancel(self, ticket):
        return lib().rve_server_cancel(self.s, ticket)

    def stats(self):
        q, a, c = ctypes.c_longlong(), ctypes.c_longlong(), ctypes.c_longlong()
        b = _SZ()
        _check(lib().rve_server_stats(self.s, ctypes.byref(q), ctypes.byref(a), ctypes.byref(c), ctypes.byref(b)),
               "rve_server_stats")
        return {"queued": q.value, "active": a.value, "completed": c.value, "bytes": b.value}

    def close(self):
        if self.s is not None:
            lib().rve_server_destroy(self.s)
            self.s = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ------------------------------------------------------------------ owner object

class Rve:
    """One solver handle: ``Rve(dim, n, model="neohookean", precision="fp64", **options)``."""

    def __init__(self, dim, n, model="neohookean", precision="fp64", stream=None, use_torch=True, **options):
        self.dim, self.n = int(dim), int(n)
        self.model = MODELS[model] if isinstance(model, str) else int(model)
        opt = rve_default_options()
        opt.precision = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
        for k, v in options.items():
            if k == "rho_policy" and isinstance(v, str):
                v = {"fixed": RVE_RHO_FIXED, "adaptive": RVE_RHO_ADAPTIVE}[v]
            if k == "lambda0" and isinstance(v, str):
                v = {"stress": RVE_LAMBDA0_STRESS, "zero": RVE_LAMBDA0_ZERO}[v]
            setattr(opt, k, v)
        self.opt = opt
        self._ws = None
        self.h = None
        if stream is None and use_torch:
            import torch
            stream = torch.cuda.current_stream().cuda_stream
        if use_torch:
            import torch
            nbytes = self.workspace_bytes()
            self._ws = torch.empty(nbytes + 256, dtype=torch.uint8, device="cuda")
            base = self._ws.data_ptr()
            aligned = (base + 255) // 256 * 256
            rc, h = rve_create_in(self.dim, self.n, self.model, opt, stream, aligned, nbytes)
        else:
            rc, h = rve_create(self.dim, self.n, self.model, opt, stream)
        _check(rc, "rve_create")
        self.h = h

    def workspace_bytes(self):
        return rve_workspace_bytes(self.dim, self.n, self.model, self.opt)

    @property
    def grid(self):
        return (self.n,) * self.dim

    def set_material(self, phase, params, n0=None):
        ph = np.asarray(phase)
        if ph.shape != self.grid:
            raise ValueError(f"phase shape {ph.shape} != {self.grid}")
        _check(rve_set_material(self.h, ph, params, n0), "rve_set_material")

    def solve(self, Fbar, rho, tol, check=False, free=None):
        """free: optional (3, 3) boolean mask of free <F> components (rve_solve_mixed)."""
        if free is None:
            rc, info = rve_solve(self.h, Fbar, rho, tol)
        else:
            rc, info = rve_solve_mixed(self.h, Fbar, free, rho, tol)
        if rc not in (RVE_OK, RVE_E_NOT_CONVERGED) or (check and rc != RVE_OK):
            raise RveError(rc, "rve_solve")
        return info

    def solve_path(self, Fbars, rho, tol, free=None):
        """Loading path (rve_solve_path): Fbars of shape (steps, 3, 3); returns (S, Fbar, infos)
        with S and Fbar of shape (steps, 3, 3)."""
        fb = np.ascontiguousarray(np.asarray(Fbars, dtype=np.float64).reshape(-1, 9))
        steps = fb.shape[0]
        S = np.zeros((steps, 9))
        Fo = np.zeros((steps, 9))
        infos = (rve_solve_info * steps)()
        mask = 0 if free is None else free_mask_bits(free)
        rc = lib().rve_solve_path(self.h, _dptr(fb), steps, mask, float(rho), float(tol), _dptr(S), _dptr(Fo), infos)
        if rc not in (RVE_OK, RVE_E_NOT_CONVERGED):
            raise RveError(rc, "rve_solve_path")
        return S.reshape(steps, 3, 3), Fo.reshape(steps, 3, 3), list(infos)

    def bloch(self, k, rho, tol, max_iter, p0=None, seed=0):
        """Modulus of stability beta_k of the resident state (rve_bloch).  p0 defaults to
        synth.bloch_start(n, dim, seed).  Returns (info, p, history)."""
        if p0 is None:
            from . import synth
            p0 = synth.bloch_start(self.n, self.dim, seed)
        rc, info, p, hist = rve_bloch(self.h, k, p0, rho, tol, max_iter)
        if rc not in (RVE_OK, RVE_E_NOT_CONVERGED):
            raise RveError(rc, "rve_bloch")
        return info, p, hist

    def macro_gradient(self):
        rc, F = rve_macro_gradient(self.h)
        _check(rc, "rve_macro_gradient")
        return F

    def stress(self):
        rc, S = rve_stress(self.h)
        _check(rc, "rve_stress")
        return S[: self.dim, : self.dim].copy()

    def mean_lambda(self):
        rc, S = rve_mean_lambda(self.h)
        _check(rc, "rve_mean_lambda")
        return S[: self.dim, : self.dim].copy()

    def _shape(self, which):
        d = self.dim
        if which in (RVE_FIELD_F, RVE_FIELD_LAMBDA):
            return (d, d) + self.grid
        if which == RVE_FIELD_U:
            return (d,) + self.grid
        return (3,) + self.grid

    def get_field(self, which):
        out = np.empty(self._shape(which))
        _check(rve_get_field(self.h, which, out), "rve_get_field")
        return out

    def set_field(self, which, arr):
        a = np.asarray(arr, dtype=np.float64)
        if a.shape != self._shape(which):
            raise ValueError(f"field shape {a.shape} != {self._shape(which)}")
        _check(rve_set_field(self.h, which, a), "rve_set_field")

    def state(self):
        st = {"F": self.get_field(RVE_FIELD_F), "Lam": self.get_field(RVE_FIELD_LAMBDA),
              "u": self.get_field(RVE_FIELD_U)}
        if self.model == RVE_LCE:
            st["n"] = self.get_field(RVE_FIELD_N)
        return st

    def set_state(self, st):
        self.set_field(RVE_FIELD_F, st["F"])
        self.set_field(RVE_FIELD_LAMBDA, st["Lam"])
        self.set_field(RVE_FIELD_U, st["u"])
        if self.model == RVE_LCE:
            self.set_field(RVE_FIELD_N, st["n"])

    def reset(self):
        _check(rve_reset(self.h), "rve_reset")

    def history(self, cap=None):
        cnt, hst = rve_history(self.h, cap or (self.opt.max_iter + 1))
        if cnt < 0:
            raise RveError(cnt, "rve_history")
        return hst

    def history_local(self, cap=None):
        """r_l of the local step fused with each check (entry i: Step 1 of iteration i + 2)."""
        cnt, rl = rve_history_local(self.h, cap or (self.opt.max_iter + 1))
        if cnt < 0:
            raise RveError(cnt, "rve_history_local")
        return rl

    def set_profiling(self, on):
        _check(rve_set_profiling(self.h, on), "rve_set_profiling")

    def kernel_times(self):
        """{precision: {class: (total_ms, launches)}} for classes with launches."""
        out = {}
        for name, f in (("fp64", True), ("fp32", False)):
            rc, ms, n = rve_kernel_times(self.h, f)
            if rc < 0:
                raise RveError(rc, "rve_kernel_times")
            out[name] = {KCLASS_NAMES[c]: (float(ms[c]), int(n[c])) for c in range(len(KCLASS_NAMES)) if n[c]}
        return out

    def close(self):
        if self.h is not None:
            rve_destroy(self.h)
            self.h = None
        self._ws = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
