"""ctypes binding of libtpcg (include/tpcg.h): argument marshalling only.

Every function here has the name of the C entry point it calls and does no
arithmetic of the method.  ``Plan`` is a small convenience wrapper that
passes PyTorch tensors' device pointers and the current CUDA stream.

There is no CPU fallback: if ``libtpcg.so`` has not been built (see
``paper_2501_03377_gb300.build``) every call raises.
"""
from __future__ import annotations

import ctypes
import os

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libtpcg.so")

TPCG_OK = 0
TPCG_ERR_INVALID_ARG = 1
TPCG_ERR_OOM = 2
TPCG_ERR_CUDA = 3
TPCG_ERR_NOT_CONVERGED = 4
TPCG_ERR_BREAKDOWN = 5
TPCG_ERR_TIMEOUT = 6
TPCG_ERR_UNSUPPORTED = 7
TPCG_ERR_EIGENBASIS = 8
TPCG_ERR_ADMISSION = 9
TPCG_PENDING = 10
TPCG_ERR_UNKNOWN_TICKET = 11
TPCG_ERR_CANCELLED = 12

TPCG_BC_P, TPCG_BC_D, TPCG_BC_N, TPCG_BC_DN, TPCG_BC_ND = 0, 1, 2, 3, 4
BC = {"P": TPCG_BC_P, "D": TPCG_BC_D, "N": TPCG_BC_N, "DN": TPCG_BC_DN, "ND": TPCG_BC_ND}
TPCG_FP64 = 0
TPCG_MIXED_TF32 = 1
TPCG_MIXED_BF16 = 2
TPCG_MIXED_FP16 = 3
TPCG_MIXED_BF16X3 = 4
PREC = {"fp64": TPCG_FP64, "tf32": TPCG_MIXED_TF32, "bf16": TPCG_MIXED_BF16, "fp16": TPCG_MIXED_FP16,
        "bf16x3": TPCG_MIXED_BF16X3}
TPCG_ZERO_GUESS = 1
TPCG_PRECOND_PINV = 0
TPCG_PRECOND_NONE = 1
TPCG_PRECOND_JACOBI = 2
TPCG_OPT_DEFER_U = 1
TPCG_OPT_FUSE_G = 2
TPCG_OPT_SLICES = 3
TPCG_OPT_GRAPHS = 4
TPCG_OPT_SWEEP_GRAIN = 5
TPCG_REQ_BORROW_HOST = 1
TPCG_REQ_BORROW_DEVICE = 2


class tpcg_info(ctypes.Structure):
    _fields_ = [
        ("status", ctypes.c_int),
        ("iters", ctypes.c_int),
        ("precond_applies", ctypes.c_int),
        ("prec", ctypes.c_int),
        ("rel_res_true", ctypes.c_double),
        ("rel_res_recur", ctypes.c_double),
        ("eta_norm", ctypes.c_double),
        ("removed_mean", ctypes.c_double),
        ("null_component", ctypes.c_double),
        ("checks", ctypes.c_int),
    ]

    def as_dict(self):
        return {name: getattr(self, name) for name, _ in self._fields_}


class tpcg_cg_scalars(ctypes.Structure):
    _fields_ = [("iter", ctypes.c_int), ("alpha", ctypes.c_double), ("beta", ctypes.c_double),
                ("rho", ctypes.c_double), ("wp", ctypes.c_double), ("rr", ctypes.c_double),
                ("sum_r", ctypes.c_double), ("mean_z", ctypes.c_double), ("lp_shift", ctypes.c_int),
                ("direction_exponent", ctypes.c_int)]

    def as_dict(self):
        return {name: getattr(self, name) for name, _ in self._fields_}


class tpcg_tune_result(ctypes.Structure):
    _fields_ = [("slices", ctypes.c_int), ("fuse_g", ctypes.c_int), ("us_per_apply", ctypes.c_double),
                ("candidates", ctypes.c_int), ("from_cache", ctypes.c_int)]

    def as_dict(self):
        return {name: getattr(self, name) for name, _ in self._fields_}


class tpcg_kernel_stat(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 24), ("launches", ctypes.c_ulonglong), ("total_ms", ctypes.c_double)]


class tpcg_request(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int), ("bc", ctypes.c_int * 3),
                ("h", ctypes.c_double * 3), ("prec", ctypes.c_int), ("session", ctypes.c_ulonglong),
                ("eta", ctypes.c_void_p), ("tol", ctypes.c_double), ("maxit", ctypes.c_int),
                ("flags", ctypes.c_uint)]


class tpcg_server_stats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_ulonglong), ("completed", ctypes.c_ulonglong), ("failed", ctypes.c_ulonglong),
                ("rejected", ctypes.c_ulonglong), ("queued", ctypes.c_int), ("running", ctypes.c_int),
                ("device_bytes", ctypes.c_size_t), ("p50_ms", ctypes.c_double), ("p99_ms", ctypes.c_double),
                ("mean_ms", ctypes.c_double), ("elapsed_s", ctypes.c_double)]

    def as_dict(self):
        return {name: getattr(self, name) for name, _ in self._fields_}


class tpcg_request_timing(ctypes.Structure):
    _fields_ = [("ticket", ctypes.c_ulonglong), ("session", ctypes.c_ulonglong), ("nx", ctypes.c_int),
                ("ny", ctypes.c_int), ("nz", ctypes.c_int), ("prec", ctypes.c_int), ("status", ctypes.c_int),
                ("iters", ctypes.c_int), ("plan_built", ctypes.c_int), ("queue_ms", ctypes.c_double),
                ("build_ms", ctypes.c_double), ("solve_ms", ctypes.c_double), ("copy_ms", ctypes.c_double),
                ("total_ms", ctypes.c_double)]

    def as_dict(self):
        return {name: getattr(self, name) for name, _ in self._fields_}


_P = ctypes.c_void_p
_D = ctypes.c_double
_I = ctypes.c_int
_SIGS = {
    "tpcg_plan_create": (_I, [_I, _I, _I, ctypes.POINTER(_I), ctypes.POINTER(_D), _I, _P, ctypes.POINTER(_P)]),
    "tpcg_plan_destroy": (_I, [_P]),
    "tpcg_plan_set_stream": (_I, [_P, _P]),
    "tpcg_plan_device_bytes": (_I, [_P, ctypes.POINTER(ctypes.c_size_t)]),
    "tpcg_solve": (_I, [_P, _P, _P, _D, _I, ctypes.c_uint, ctypes.POINTER(tpcg_info)]),
    "tpcg_solve_host": (_I, [_P, _P, _P, _D, _I, ctypes.c_uint, ctypes.POINTER(tpcg_info)]),
    "tpcg_solve_host_stream": (_I, [_P, _I, ctypes.POINTER(_P), ctypes.POINTER(_P), _D, _I, ctypes.c_uint,
                                    ctypes.POINTER(tpcg_info)]),
    "tpcg_solve_batched": (_I, [ctypes.POINTER(_P), _I, ctypes.POINTER(_I), ctypes.POINTER(_P), ctypes.POINTER(_P),
                                ctypes.POINTER(_D), _I, ctypes.c_uint, ctypes.POINTER(tpcg_info)]),
    "tpcg_precond_apply": (_I, [_P, _P, _P]),
    "tpcg_apply_laplacian": (_I, [_P, _P, _P]),
    "tpcg_rhs_add_bc": (_I, [_P, _P, ctypes.POINTER(_D)]),
    "tpcg_efield": (_I, [_P, _P, ctypes.POINTER(_D), _P, _P, _P]),
    "tpcg_plan_set_precond": (_I, [_P, _I, _I, _D]),
    "tpcg_plan_set_option": (_I, [_P, _I, _I]),
    "tpcg_plan_eigenpairs": (_I, [_P, _I, ctypes.POINTER(_D), ctypes.POINTER(_D)]),
    "tpcg_plan_cg_scalars": (_I, [_P, ctypes.POINTER(tpcg_cg_scalars)]),
    "tpcg_plan_autotune": (_I, [_P, ctypes.c_char_p, _I, ctypes.POINTER(tpcg_tune_result)]),
    "tpcg_plan_cg_vectors": (_I, [_P, _P, _P, _P]),
    "tpcg_plan_launch_count": (_I, [_P, ctypes.POINTER(ctypes.c_ulonglong)]),
    "tpcg_plan_precond_launches": (_I, [_P, ctypes.POINTER(ctypes.c_int)]),
    "tpcg_profile_begin": (_I, [_P]),
    "tpcg_profile_end": (_I, [_P, ctypes.POINTER(tpcg_kernel_stat), _I, ctypes.POINTER(_I)]),
    "tpcg_residual_norms_noalloc": (_I, [_I, _I, _I, ctypes.POINTER(_I), ctypes.POINTER(_D), _P, _P, _P, _P]),
    "tpcg_server_create": (_I, [ctypes.c_size_t, _I, ctypes.POINTER(_P)]),
    "tpcg_server_submit": (_I, [_P, ctypes.POINTER(tpcg_request), ctypes.POINTER(ctypes.c_ulonglong)]),
    "tpcg_server_poll": (_I, [_P, ctypes.c_ulonglong, _P, ctypes.POINTER(tpcg_info)]),
    "tpcg_server_wait": (_I, [_P, ctypes.c_ulonglong, _D, _P, ctypes.POINTER(tpcg_info)]),
    "tpcg_server_get_stats": (_I, [_P, ctypes.POINTER(tpcg_server_stats)]),
    "tpcg_server_get_timings": (_I, [_P, ctypes.POINTER(tpcg_request_timing), _I, ctypes.POINTER(_I)]),
    "tpcg_server_reset_stats": (_I, [_P]),
    "tpcg_server_destroy": (_I, [_P]),
    "tpcg_strerror": (ctypes.c_char_p, [_I]),
}
_lib = None


def lib():
    """Load libtpcg.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"libtpcg.so not built ({LIB_PATH}); run paper_2501_03377_gb300.build.build()")
        handle = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in _SIGS.items():
            fn = getattr(handle, name)
            fn.restype = res
            fn.argtypes = args
        _lib = handle
    return _lib


def declared_symbols():
    return list(_SIGS)


class TpcgError(RuntimeError):
    def __init__(self, status, what=""):
        self.status = status
        super().__init__(f"{what}: {tpcg_strerror(status)} ({status})")


def tpcg_strerror(status: int) -> str:
    return lib().tpcg_strerror(int(status)).decode()


def tpcg_plan_create(nx, ny, nz, bc, h, prec, stream):
    bc_arr = (_I * 3)(*[BC[b] if isinstance(b, str) else int(b) for b in bc])
    h_arr = (_D * 3)(*[float(v) for v in h])
    out = _P()
    st = lib().tpcg_plan_create(int(nx), int(ny), int(nz), bc_arr, h_arr, int(prec), _P(stream), ctypes.byref(out))
    return st, out


def tpcg_plan_destroy(plan):
    return lib().tpcg_plan_destroy(plan)


def tpcg_plan_set_stream(plan, stream):
    return lib().tpcg_plan_set_stream(plan, _P(stream))


def tpcg_plan_device_bytes(plan):
    v = ctypes.c_size_t()
    st = lib().tpcg_plan_device_bytes(plan, ctypes.byref(v))
    return st, v.value


def tpcg_solve(plan, eta_ptr, ups_ptr, tol, maxit, flags):
    info = tpcg_info()
    st = lib().tpcg_solve(plan, _P(eta_ptr), _P(ups_ptr), float(tol), int(maxit), int(flags), ctypes.byref(info))
    return st, info


def tpcg_solve_host(plan, eta_ptr, ups_ptr, tol, maxit, flags):
    info = tpcg_info()
    st = lib().tpcg_solve_host(plan, _P(eta_ptr), _P(ups_ptr), float(tol), int(maxit), int(flags), ctypes.byref(info))
    return st, info


def tpcg_solve_host_stream(plan, eta_ptrs, ups_ptrs, tol, maxit, flags):
    n = len(eta_ptrs)
    infos = (tpcg_info * max(1, n))()
    ea = (_P * max(1, n))(*[_P(x) for x in eta_ptrs])
    ua = (_P * max(1, n))(*[_P(x) for x in ups_ptrs])
    st = lib().tpcg_solve_host_stream(plan, n, ea, ua, float(tol), int(maxit), int(flags), infos)
    return st, [infos[i] for i in range(n)]


def tpcg_solve_batched(plans, nrhs, eta_ptrs, ups_ptrs, tols, maxit, flags):
    n = len(plans)
    total = sum(nrhs)
    infos = (tpcg_info * max(1, total))()
    st = lib().tpcg_solve_batched((_P * n)(*plans), n, (_I * n)(*nrhs), (_P * n)(*eta_ptrs), (_P * n)(*ups_ptrs),
                                  (_D * n)(*tols), int(maxit), int(flags), infos)
    return st, [infos[i].as_dict() for i in range(total)]


def tpcg_precond_apply(plan, r_ptr, z_ptr):
    return lib().tpcg_precond_apply(plan, _P(r_ptr), _P(z_ptr))


def tpcg_apply_laplacian(plan, x_ptr, w_ptr):
    return lib().tpcg_apply_laplacian(plan, _P(x_ptr), _P(w_ptr))


def tpcg_plan_set_option(plan, option, value):
    return lib().tpcg_plan_set_option(plan, int(option), int(value))


def tpcg_plan_set_precond(plan, kind, p=3, omega=1.3):
    return lib().tpcg_plan_set_precond(plan, int(kind), int(p), float(omega))


def tpcg_efield(plan, ups_ptr, bval, ex_ptr, ey_ptr, ez_ptr):
    arr = None if bval is None else (_D * 6)(*[float(v) for v in bval])
    return lib().tpcg_efield(plan, _P(ups_ptr), arr, _P(ex_ptr), _P(ey_ptr), _P(ez_ptr))


def tpcg_rhs_add_bc(plan, eta_ptr, bval):
    arr = (_D * 6)(*[float(v) for v in bval])
    return lib().tpcg_rhs_add_bc(plan, _P(eta_ptr), arr)


def tpcg_plan_eigenpairs(plan, axis, length):
    lam = (_D * length)()
    V = (_D * (length * length))()
    st = lib().tpcg_plan_eigenpairs(plan, int(axis), lam, V)
    return st, list(lam), list(V)


def tpcg_plan_autotune(plan, cache_path=None, applies=5):
    out = tpcg_tune_result()
    st = lib().tpcg_plan_autotune(plan, cache_path.encode() if cache_path else None, int(applies), ctypes.byref(out))
    return st, out.as_dict()


def tpcg_plan_cg_scalars(plan):
    out = tpcg_cg_scalars()
    st = lib().tpcg_plan_cg_scalars(plan, ctypes.byref(out))
    return st, out.as_dict()


def tpcg_plan_cg_vectors(plan, r_ptr, z_ptr, p_ptr):
    return lib().tpcg_plan_cg_vectors(plan, _P(r_ptr), _P(z_ptr), _P(p_ptr))


def tpcg_plan_launch_count(plan):
    v = ctypes.c_ulonglong()
    st = lib().tpcg_plan_launch_count(plan, ctypes.byref(v))
    return st, v.value


def tpcg_plan_precond_launches(plan):
    v = ctypes.c_int()
    st = lib().tpcg_plan_precond_launches(plan, ctypes.byref(v))
    return st, v.value


def tpcg_profile_begin(plan):
    return lib().tpcg_profile_begin(plan)


def tpcg_profile_end(plan, max_stats=16):
    arr = (tpcg_kernel_stat * max_stats)()
    n = _I()
    st = lib().tpcg_profile_end(plan, arr, max_stats, ctypes.byref(n))
    out = {arr[i].name.decode(): {"launches": arr[i].launches, "total_ms": arr[i].total_ms} for i in range(n.value)}
    return st, out


def tpcg_residual_norms_noalloc(nx, ny, nz, bc, h, eta_ptr, ups_ptr, out_ptr, stream):
    bc_arr = (_I * 3)(*[BC[b] if isinstance(b, str) else int(b) for b in bc])
    h_arr = (_D * 3)(*[float(v) for v in h])
    return lib().tpcg_residual_norms_noalloc(int(nx), int(ny), int(nz), bc_arr, h_arr, _P(eta_ptr), _P(ups_ptr),
                                             _P(out_ptr), _P(stream))


def tpcg_server_create(hbm_budget, max_slots):
    out = _P()
    st = lib().tpcg_server_create(int(hbm_budget), int(max_slots), ctypes.byref(out))
    return st, out


def tpcg_server_submit(server, req):
    t = ctypes.c_ulonglong()
    st = lib().tpcg_server_submit(server, ctypes.byref(req), ctypes.byref(t))
    return st, t.value


def tpcg_server_poll(server, ticket, ups_ptr):
    info = tpcg_info()
    st = lib().tpcg_server_poll(server, ctypes.c_ulonglong(ticket), _P(ups_ptr), ctypes.byref(info))
    return st, info


def tpcg_server_wait(server, ticket, timeout_s, ups_ptr):
    info = tpcg_info()
    st = lib().tpcg_server_wait(server, ctypes.c_ulonglong(ticket), float(timeout_s), _P(ups_ptr),
                                ctypes.byref(info))
    return st, info


def tpcg_server_get_timings(server):
    n = _I()
    st = lib().tpcg_server_get_timings(server, None, 0, ctypes.byref(n))
    if st != TPCG_OK or n.value == 0:
        return st, []
    arr = (tpcg_request_timing * n.value)()
    st = lib().tpcg_server_get_timings(server, arr, n.value, ctypes.byref(n))
    return st, [arr[i].as_dict() for i in range(n.value)]


def tpcg_server_get_stats(server):
    out = tpcg_server_stats()
    st = lib().tpcg_server_get_stats(server, ctypes.byref(out))
    return st, out


def tpcg_server_reset_stats(server):
    return lib().tpcg_server_reset_stats(server)


def tpcg_server_destroy(server):
    return lib().tpcg_server_destroy(server)


class Server:
    """Owns a tpcg_server; right-hand sides and solutions are host numpy float64 arrays (nz, ny, nx)."""

    def __init__(self, hbm_budget=0, max_slots=8):
        st, h = tpcg_server_create(hbm_budget, max_slots)
        if st != TPCG_OK:
            raise TpcgError(st, "tpcg_server_create")
        self.handle = h
        self.shapes = {}

    def submit(self, eta, bcs, h=(1.0, 1.0, 1.0), prec="fp16", session=0, tol=1e-10, maxit=60, borrow=False):
        """eta: numpy array (copied by the server), or with borrow=True a torch tensor (pinned host or
        CUDA) that the caller keeps alive and unchanged until the result is taken."""
        import numpy as np

        flags = 0
        if borrow:
            nz, ny, nx = eta.shape
            ptr = eta.data_ptr()
            flags = TPCG_REQ_BORROW_DEVICE if eta.is_cuda else TPCG_REQ_BORROW_HOST
        else:
            eta = np.ascontiguousarray(eta, dtype=np.float64)
            nz, ny, nx = eta.shape
            ptr = eta.ctypes.data
        req = tpcg_request()
        req.nx, req.ny, req.nz = nx, ny, nz
        for m in range(3):
            b = bcs[m] if m < len(bcs) else "P"
            req.bc[m] = BC[b] if isinstance(b, str) else int(b)
            req.h[m] = float(h[m])
        req.prec = PREC[prec] if isinstance(prec, str) else int(prec)
        req.session = int(session)
        req.eta = ptr
        req.tol = float(tol)
        req.maxit = int(maxit)
        req.flags = flags
        st, t = tpcg_server_submit(self.handle, req)
        if st != TPCG_OK:
            raise TpcgError(st, "tpcg_server_submit")
        self.shapes[t] = tuple(eta.shape)
        return t

    def _result(self, fn, ticket, *args, want=True):
        import numpy as np

        out = np.empty(self.shapes[ticket]) if want else None
        st, info = fn(self.handle, ticket, *args, out.ctypes.data if want else None)
        if st == TPCG_PENDING:
            return st, None, None
        self.shapes.pop(ticket, None)
        return st, out, info.as_dict()

    def poll(self, ticket, want=True):
        """(status, solution or None while pending, info); want=False: report only, no copy of the solution."""
        return self._result(tpcg_server_poll, ticket, want=want)

    def wait(self, ticket, timeout_s=-1.0, want=True):
        return self._result(tpcg_server_wait, ticket, timeout_s, want=want)

    def stats(self):
        return tpcg_server_get_stats(self.handle)[1].as_dict()

    def timings(self):
        """Per-request latency breakdown (queue, plan build, solve, copy) of the finished requests."""
        return tpcg_server_get_timings(self.handle)[1]

    def reset_stats(self):
        tpcg_server_reset_stats(self.handle)

    def close(self):
        if getattr(self, "handle", None):
            tpcg_server_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ---------------------------------------------------------------------------
class Plan:
    """Owns a tpcg_plan; tensors are torch float64 CUDA tensors of shape (nz, ny, nx)."""

    def __init__(self, nx, ny, nz, bcs, h=(1.0, 1.0, 1.0), prec="fp64", stream=None):
        import torch

        if stream is None:
            stream = torch.cuda.current_stream().cuda_stream
        self.shape = (nz, ny, nx)
        self.nx, self.ny, self.nz = nx, ny, nz
        self.device = torch.device("cuda", torch.cuda.current_device())
        self.prec = PREC[prec] if isinstance(prec, str) else int(prec)
        st, handle = tpcg_plan_create(nx, ny, nz, bcs, h, self.prec, stream)
        if st != TPCG_OK:
            raise TpcgError(st, "tpcg_plan_create")
        self.handle = handle

    def close(self):
        if getattr(self, "handle", None):
            tpcg_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, t):
        import torch

        if not (t.is_cuda and t.dtype == torch.float64 and t.is_contiguous() and tuple(t.shape) == self.shape):
            raise ValueError(f"expected contiguous float64 CUDA tensor of shape {self.shape}")

    def solve(self, eta, ups, tol=1e-10, maxit=100, zero_guess=False, raise_on_error=False):
        self._check(eta)
        self._check(ups)
        st, info = tpcg_solve(self.handle, eta.data_ptr(), ups.data_ptr(), tol, maxit,
                              TPCG_ZERO_GUESS if zero_guess else 0)
        if raise_on_error and st != TPCG_OK:
            raise TpcgError(st, "tpcg_solve")
        return st, info.as_dict()

    def solve_host(self, eta_host, ups_host, tol=1e-10, maxit=100, zero_guess=False):
        st, info = tpcg_solve_host(self.handle, eta_host.data_ptr(), ups_host.data_ptr(), tol, maxit,
                                   TPCG_ZERO_GUESS if zero_guess else 0)
        return st, info.as_dict()

    def solve_host_stream(self, etas_host, ups_host, tol=1e-10, maxit=100, zero_guess=False):
        """Solve for a list of host right-hand sides with the copies overlapping the solves."""
        if len(etas_host) != len(ups_host):
            raise ValueError("one solution buffer per right-hand side")
        import torch

        for t in list(etas_host) + list(ups_host):
            if t.is_cuda or t.dtype != torch.float64 or not t.is_contiguous() or tuple(t.shape) != self.shape:
                raise ValueError(f"expected contiguous float64 CPU tensors of shape {self.shape}")
        st, infos = tpcg_solve_host_stream(self.handle, [t.data_ptr() for t in etas_host],
                                           [t.data_ptr() for t in ups_host], tol, maxit,
                                           TPCG_ZERO_GUESS if zero_guess else 0)
        return st, [i.as_dict() for i in infos]

    def precond(self, r, z):
        self._check(r)
        self._check(z)
        st = tpcg_precond_apply(self.handle, r.data_ptr(), z.data_ptr())
        if st != TPCG_OK:
            raise TpcgError(st, "tpcg_precond_apply")

    def laplacian(self, x, w):
        self._check(x)
        self._check(w)
        st = tpcg_apply_laplacian(self.handle, x.data_ptr(), w.data_ptr())
        if st != TPCG_OK:
            raise TpcgError(st, "tpcg_apply_laplacian")

    def set_option(self, option, value):
        """Plan option: TPCG_OPT_DEFER_U (1: record U += alpha P and form U before each check),
        TPCG_OPT_FUSE_G (0: the products around G in separate launches), TPCG_OPT_SLICES (0: one
        launch per mode product instead of the frontal-slice launches), TPCG_OPT_GRAPHS (0: launch
        every kernel directly instead of replaying captured launch sequences) or TPCG_OPT_SWEEP_GRAIN
        (1..64, default 4: least work per block of the sweeps; larger for many small plans at once)."""
        st = tpcg_plan_set_option(self.handle, option, value)
        if st != TPCG_OK:
            raise TpcgError(st, "tpcg_plan_set_option")

    def set_precond(self, kind, p=3, omega=1.3):
        """Choose the preconditioner ("pinv", "none" or "jacobi"); see tpcg_plan_set_precond."""
        code = {"pinv": TPCG_PRECOND_PINV, "none": TPCG_PRECOND_NONE, "jacobi": TPCG_PRECOND_JACOBI}[kind]
        st = tpcg_plan_set_precond(self.handle, code, p, omega)
        if st:
            raise TpcgError(st, "tpcg_plan_set_precond")

    def efield(self, ups, ex, ey, ez=None, bval=None):
        """Electric field -grad(ups) into ex, ey (and ez in 3D); see tpcg_efield."""
        for t in (ups, ex, ey) + ((ez,) if ez is not None else ()):
            self._check(t)
        st = tpcg_efield(self.handle, ups.data_ptr(), bval, ex.data_ptr(), ey.data_ptr(),
                         ez.data_ptr() if ez is not None else 0)
        if st:
            raise TpcgError(st, "tpcg_efield")

    def rhs_add_bc(self, eta, bval):
        self._check(eta)
        st = tpcg_rhs_add_bc(self.handle, eta.data_ptr(), bval)
        if st != TPCG_OK:
            raise TpcgError(st, "tpcg_rhs_add_bc")

    def eigenpairs(self, axis):
        length = (self.nx, self.ny, self.nz)[axis]
        st, lam, V = tpcg_plan_eigenpairs(self.handle, axis, length)
        if st != TPCG_OK:
            raise TpcgError(st, "tpcg_plan_eigenpairs")
        return lam, V

    def launch_count(self):
        return tpcg_plan_launch_count(self.handle)[1]

    def autotune(self, cache_path=None, applies=5):
        """Time the preconditioner's launch sequences and keep the fastest (tpcg_plan_autotune)."""
        st, d = tpcg_plan_autotune(self.handle, cache_path, applies)
        if st != TPCG_OK:
            raise TpcgError(st, "tpcg_plan_autotune")
        return d

    def cg_scalars(self):
        """Device scalars of the most recent CG iteration (see tpcg_plan_cg_scalars)."""
        st, d = tpcg_plan_cg_scalars(self.handle)
        if st != TPCG_OK:
            raise TpcgError(st, "tpcg_plan_cg_scalars")
        return d

    def cg_vectors(self):
        """FP64 copies (torch tensors) of the plan's current R, Z and last direction P."""
        import torch

        shape = (self.nz, self.ny, self.nx)
        R, Z, P = (torch.empty(shape, dtype=torch.float64, device=self.device) for _ in range(3))
        st = tpcg_plan_cg_vectors(self.handle, R.data_ptr(), Z.data_ptr(), P.data_ptr())
        if st != TPCG_OK:
            raise TpcgError(st, "tpcg_plan_cg_vectors")
        return R, Z, P

    def precond_launches(self):
        """Tensor-core launches per preconditioner application (0 for the FP64 form)."""
        return tpcg_plan_precond_launches(self.handle)[1]

    def profile_begin(self):
        tpcg_profile_begin(self.handle)

    def profile_end(self):
        st, stats = tpcg_profile_end(self.handle)
        if st != TPCG_OK:
            raise TpcgError(st, "tpcg_profile_end")
        return stats

    def device_bytes(self):
        return tpcg_plan_device_bytes(self.handle)[1]
