"""Thin ctypes binding of the C ABI in ``include/hh.h`` (argument marshalling only).

Every step of the solver runs in ``libhh.so``; this module passes torch device
pointers, sizes and the current CUDA stream across the ABI and turns status codes
into exceptions.  There is no fallback: if the library is missing or was built for
another machine, loading fails loudly.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np
import torch

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libhh.so")

HH_OK, HH_NOT_CONVERGED = 0, 1
HH_C128, HH_C64 = 0, 1
SOMMERFELD, DIRICHLET = 0, 1
OP = {"K": 0, "M": 1, "MGAMMA": 2, "AL": 3, "AR": 4, "B": 5, "BHAT": 6}

EXPORTED = (
    "hh_options_default", "hh_footprint_bytes", "hh_create_problem", "hh_destroy", "hh_solve",
    "hh_solve_host", "hh_level_nodes", "hh_apply", "hh_jacobi", "hh_residual_restrict",
    "hh_prolong_correct", "hh_vcycle", "hh_hss_rhs", "hh_precondition", "hh_load_vector", "hh_dot",
    "hh_multidot_noalloc", "hh_status_string", "hh_last_error",
)


class Grid(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int), ("n", ctypes.c_int)]


class Options(ctypes.Structure):
    _fields_ = [
        ("theta", ctypes.c_double), ("levels", ctypes.c_int), ("nu_pre", ctypes.c_int),
        ("nu_post", ctypes.c_int), ("nu_coarse", ctypes.c_int), ("cycles_per_hss", ctypes.c_int),
        ("omega", ctypes.c_double), ("restart", ctypes.c_int), ("max_outer", ctypes.c_int),
        ("precision", ctypes.c_int), ("use_graphs", ctypes.c_int), ("use_pdl", ctypes.c_int),
        ("coarse_cluster_nodes", ctypes.c_int), ("tile_rows", ctypes.c_int),
    ]


class Info(ctypes.Structure):
    _fields_ = [
        ("outer_its", ctypes.c_int), ("hss_its", ctypes.c_longlong), ("vcycles", ctypes.c_longlong),
        ("rel_residual", ctypes.c_double), ("seconds", ctypes.c_double), ("device_bytes", ctypes.c_size_t),
        ("kernel_launches", ctypes.c_longlong),
    ]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class HHError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"hh status {status}: {msg}")
        self.status = status


_lib = None


def load_library(path: str = LIB_PATH) -> ctypes.CDLL:
    """Load libhh.so (built by ``__graft_entry__.build()``) and declare its signatures."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build it with __graft_entry__.build()")
    lib = ctypes.CDLL(path)
    P, I, D, V = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, None
    sig = {
        "hh_options_default": (V, [ctypes.POINTER(Options)]),
        "hh_footprint_bytes": (ctypes.c_size_t, [ctypes.POINTER(Grid), ctypes.POINTER(Options)]),
        "hh_create_problem": (I, [ctypes.POINTER(Grid), D, D, D, ctypes.POINTER(ctypes.c_int),
                                  ctypes.POINTER(Options), P, ctypes.POINTER(P)]),
        "hh_destroy": (V, [P]),
        "hh_solve": (I, [P, P, D, P, P, ctypes.POINTER(Info)]),
        "hh_solve_host": (I, [P, P, D, P, ctypes.POINTER(Info)]),
        "hh_level_nodes": (ctypes.c_longlong, [P, I]),
        "hh_apply": (I, [P, I, I, I, P, P]),
        "hh_jacobi": (I, [P, I, I, P, P, P]),
        "hh_residual_restrict": (I, [P, I, I, P, P, P]),
        "hh_prolong_correct": (I, [P, I, I, P, P]),
        "hh_vcycle": (I, [P, I, P, P]),
        "hh_hss_rhs": (I, [P, I, P, P, P]),
        "hh_precondition": (I, [P, P, P]),
        "hh_load_vector": (I, [P, P, P]),
        "hh_dot": (I, [P, P, P, ctypes.POINTER(ctypes.c_double)]),
        "hh_multidot_noalloc": (I, [P, ctypes.c_longlong, I, P, ctypes.c_longlong, P, P]),
        "hh_status_string": (ctypes.c_char_p, [I]),
        "hh_last_error": (ctypes.c_char_p, []),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def _check(status, allow_not_converged=False):
    if status == HH_OK or (allow_not_converged and status == HH_NOT_CONVERGED):
        return status
    lib = load_library()
    raise HHError(status, f"{lib.hh_status_string(status).decode()}: {lib.hh_last_error().decode()}")


def default_options(**kw) -> Options:
    o = Options()
    load_library().hh_options_default(ctypes.byref(o))
    for k, v in kw.items():
        if not hasattr(o, k):
            raise KeyError(k)
        setattr(o, k, v)
    return o


def footprint_bytes(dim: int, n: int, options: Options | None = None) -> int:
    o = options or default_options()
    return int(load_library().hh_footprint_bytes(ctypes.byref(Grid(dim, n)), ctypes.byref(o)))


def _ptr(t):
    if t is None:
        return None
    if not t.is_cuda or not t.is_contiguous():
        raise ValueError("vectors must be contiguous CUDA tensors")
    return ctypes.c_void_p(t.data_ptr())


def _prec_of(t):
    if t.dtype == torch.complex64:
        return HH_C64
    if t.dtype == torch.complex128:
        return HH_C128
    raise TypeError("vectors must be complex64 or complex128")


class Problem:
    """One Helmholtz problem: grid, wavenumber k, delta, delta_hat, boundary tags, options."""

    def __init__(self, dim, n, k, delta, delta_hat, bc, options: Options | None = None, stream=None):
        lib = load_library()
        self.dim, self.n, self.k = dim, n, k
        self.options = options or default_options()
        bc = list(bc) + [0] * (6 - len(bc))
        arr = (ctypes.c_int * 6)(*bc)
        s = stream if stream is not None else torch.cuda.current_stream()
        self._stream = s
        handle = ctypes.c_void_p(s.cuda_stream)
        out = ctypes.c_void_p()
        _check(lib.hh_create_problem(ctypes.byref(Grid(dim, n)), float(k), float(delta), float(delta_hat),
                                     arr, ctypes.byref(self.options), handle, ctypes.byref(out)))
        self._p = out
        self._lib = lib

    def close(self):
        if getattr(self, "_p", None):
            self._lib.hh_destroy(self._p)
            self._p = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def nodes(self, level=0) -> int:
        return int(self._lib.hh_level_nodes(self._p, level))

    def zeros(self, level=0, dtype=torch.complex128):
        return torch.zeros(self.nodes(level), dtype=dtype, device="cuda")

    # -- solver ------------------------------------------------------------
    def solve(self, rhs, tol=1e-8, x0=None, u=None):
        u = torch.empty_like(rhs) if u is None else u
        info = Info()
        st = self._lib.hh_solve(self._p, _ptr(rhs), float(tol), _ptr(u), _ptr(x0), ctypes.byref(info))
        _check(st, allow_not_converged=True)
        return u, info

    def solve_host(self, rhs: np.ndarray, tol=1e-8, out: np.ndarray | None = None):
        rhs = np.ascontiguousarray(rhs, dtype=np.complex128)
        out = np.empty_like(rhs) if out is None else out
        info = Info()
        st = self._lib.hh_solve_host(self._p, rhs.ctypes.data_as(ctypes.c_void_p), float(tol),
                                     out.ctypes.data_as(ctypes.c_void_p), ctypes.byref(info))
        _check(st, allow_not_converged=True)
        return out, info

    # -- building blocks ------------------------------------------------------
    def apply(self, level, op, x, y=None):
        y = torch.empty_like(x) if y is None else y
        _check(self._lib.hh_apply(self._p, level, OP[op], _prec_of(x), _ptr(x), _ptr(y)))
        return y

    def jacobi(self, level, b, x_in=None, x_out=None):
        x_out = torch.empty_like(b) if x_out is None else x_out
        _check(self._lib.hh_jacobi(self._p, level, _prec_of(b), _ptr(b), _ptr(x_in), _ptr(x_out)))
        return x_out

    def residual_restrict(self, level, b, x, rc=None):
        rc = torch.empty(self.nodes(level + 1), dtype=b.dtype, device=b.device) if rc is None else rc
        _check(self._lib.hh_residual_restrict(self._p, level, _prec_of(b), _ptr(b), _ptr(x), _ptr(rc)))
        return rc

    def prolong_correct(self, level, ec, x):
        _check(self._lib.hh_prolong_correct(self._p, level, _prec_of(x), _ptr(ec), _ptr(x)))
        return x

    def vcycle(self, b, x=None):
        x = torch.empty_like(b) if x is None else x
        _check(self._lib.hh_vcycle(self._p, _prec_of(b), _ptr(b), _ptr(x)))
        return x

    def hss_rhs(self, u, r, rhs=None):
        rhs = torch.empty_like(r) if rhs is None else rhs
        _check(self._lib.hh_hss_rhs(self._p, _prec_of(r), _ptr(u), _ptr(r), _ptr(rhs)))
        return rhs

    def precondition(self, r, z=None):
        z = torch.empty_like(r) if z is None else z
        _check(self._lib.hh_precondition(self._p, _ptr(r), _ptr(z)))
        return z

    def load_vector(self, f, b=None):
        b = torch.empty_like(f) if b is None else b
        _check(self._lib.hh_load_vector(self._p, _ptr(f), _ptr(b)))
        return b

    def dot(self, x, y) -> complex:
        out = (ctypes.c_double * 2)()
        _check(self._lib.hh_dot(self._p, _ptr(x), _ptr(y), out))
        return complex(out[0], out[1])
