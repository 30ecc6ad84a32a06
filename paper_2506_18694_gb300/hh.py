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
HH_ERR_INVALID, HH_ERR_OOM, HH_ERR_CUDA, HH_ERR_NONFINITE, HH_ERR_TIMEOUT = -1, -2, -3, -4, -5
HH_C128, HH_C64 = 0, 1
HH_OUTER_FGMRES, HH_OUTER_RICHARDSON = 0, 1
HH_SMOOTH_JACOBI, HH_SMOOTH_GMRES = 0, 1
HH_FORM_PRIMAL, HH_FORM_MIXED = 0, 1
SOMMERFELD, DIRICHLET = 0, 1
OP = {"K": 0, "M": 1, "MGAMMA": 2, "AL": 3, "AR": 4, "B": 5, "BHAT": 6}

EXPORTED = (
    "hh_options_default", "hh_footprint_bytes", "hh_footprint_batch_bytes", "hh_create_problem",
    "hh_create_batch", "hh_batch_size", "hh_autotune", "hh_set_params", "hh_prepare", "hh_destroy", "hh_solve",
    "hh_solve_host", "hh_solve_host_nodal", "hh_level_nodes", "hh_apply", "hh_jacobi", "hh_residual_restrict",
    "hh_prolong_correct", "hh_vcycle", "hh_hss_rhs", "hh_precondition", "hh_load_vector", "hh_dot",
    "hh_multidot_noalloc", "hh_server_create", "hh_server_submit", "hh_server_wait", "hh_server_get_stats",
    "hh_server_set_fallback", "hh_pack_create", "hh_pack_add", "hh_pack_run", "hh_pack_take", "hh_pack_members",
    "hh_pack_destroy", "hh_server_set_pack",
    "hh_server_destroy", "hh_status_string", "hh_last_error", "hh_sigma_dofs", "hh_vector_length",
    "hh_apply_system", "hh_set_allocation_limit",
)


class Grid(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int), ("n", ctypes.c_int)]


class Options(ctypes.Structure):
    _fields_ = [
        ("theta", ctypes.c_double), ("levels", ctypes.c_int), ("nu_pre", ctypes.c_int),
        ("nu_post", ctypes.c_int), ("nu_coarse", ctypes.c_int), ("cycles_per_hss", ctypes.c_int),
        ("omega", ctypes.c_double), ("restart", ctypes.c_int), ("max_outer", ctypes.c_int),
        ("precision", ctypes.c_int), ("use_graphs", ctypes.c_int), ("use_pdl", ctypes.c_int),
        ("coarse_cluster_nodes", ctypes.c_int), ("tile_rows", ctypes.c_int), ("autotune", ctypes.c_int),
        ("fuse_sweeps", ctypes.c_int), ("outer", ctypes.c_int), ("cycle_gamma", ctypes.c_int),
        ("tile_form", ctypes.c_int), ("smoother", ctypes.c_int), ("formulation", ctypes.c_int),
        ("persistent", ctypes.c_int), ("sync_spin_limit", ctypes.c_longlong), ("stall_cycles", ctypes.c_int),
        ("coarse_kernel", ctypes.c_int),
    ]


class Info(ctypes.Structure):
    _fields_ = [
        ("outer_its", ctypes.c_int), ("hss_its", ctypes.c_longlong), ("vcycles", ctypes.c_longlong),
        ("rel_residual", ctypes.c_double), ("seconds", ctypes.c_double), ("device_bytes", ctypes.c_size_t),
        ("kernel_launches", ctypes.c_longlong), ("fallback", ctypes.c_int),
    ]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class Request(ctypes.Structure):
    _fields_ = [("grid", Grid), ("k", ctypes.c_double), ("delta", ctypes.c_double), ("delta_hat", ctypes.c_double),
                ("bc", ctypes.c_int * 6), ("tol", ctypes.c_double), ("rhs_kind", ctypes.c_int)]


class ServerStats(ctypes.Structure):
    _fields_ = [
        ("submitted", ctypes.c_longlong), ("completed", ctypes.c_longlong), ("failed", ctypes.c_longlong),
        ("queued", ctypes.c_longlong), ("running", ctypes.c_int), ("max_concurrent", ctypes.c_int),
        ("budget", ctypes.c_size_t), ("held_bytes", ctypes.c_size_t), ("peak_bytes", ctypes.c_size_t),
        ("problems_created", ctypes.c_longlong), ("problems_reused", ctypes.c_longlong),
        ("problems_evicted", ctypes.c_longlong),
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
        "hh_footprint_batch_bytes": (ctypes.c_size_t, [ctypes.POINTER(Grid), ctypes.POINTER(Options), I]),
        "hh_create_problem": (I, [ctypes.POINTER(Grid), D, D, D, ctypes.POINTER(ctypes.c_int),
                                  ctypes.POINTER(Options), P, ctypes.POINTER(P)]),
        "hh_create_batch": (I, [ctypes.POINTER(Grid), I, ctypes.POINTER(D), ctypes.POINTER(D), ctypes.POINTER(D),
                                ctypes.POINTER(ctypes.c_int), ctypes.POINTER(Options), P, ctypes.POINTER(P)]),
        "hh_batch_size": (I, [P]),
        "hh_sigma_dofs": (ctypes.c_longlong, [ctypes.POINTER(Grid)]),
        "hh_vector_length": (ctypes.c_longlong, [P]),
        "hh_apply_system": (I, [P, P, P]),
        "hh_set_allocation_limit": (V, [ctypes.c_size_t]),
        "hh_autotune": (I, [P, I, ctypes.POINTER(ctypes.c_int)]),
        "hh_set_params": (I, [P, ctypes.POINTER(D), ctypes.POINTER(D), ctypes.POINTER(D)]),
        "hh_prepare": (I, [P]),
        "hh_server_create": (I, [I, ctypes.c_size_t, ctypes.POINTER(Options), ctypes.POINTER(P)]),
        "hh_server_submit": (I, [P, ctypes.POINTER(Request), P, P, ctypes.POINTER(ctypes.c_longlong)]),
        "hh_server_wait": (I, [P, ctypes.c_longlong, ctypes.POINTER(Info), ctypes.POINTER(D), ctypes.POINTER(D)]),
        "hh_server_get_stats": (I, [P, ctypes.POINTER(ServerStats)]),
        "hh_server_set_fallback": (I, [P, ctypes.POINTER(Options), D]),
        "hh_pack_create": (I, [I, ctypes.POINTER(P)]),
        "hh_pack_add": (I, [P, P, P, I, D, P, ctypes.POINTER(ctypes.c_int)]),
        "hh_pack_run": (I, [P, I, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)]),
        "hh_server_set_pack": (I, [P, I, I]),
        "hh_pack_take": (I, [P, I, ctypes.POINTER(Info)]),
        "hh_pack_members": (I, [P]),
        "hh_pack_destroy": (V, [P]),
        "hh_server_destroy": (V, [P]),
        "hh_destroy": (V, [P]),
        "hh_solve": (I, [P, P, D, P, P, ctypes.POINTER(Info)]),
        "hh_solve_host": (I, [P, P, D, P, ctypes.POINTER(Info)]),
        "hh_solve_host_nodal": (I, [P, P, D, P, ctypes.POINTER(Info)]),
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


def footprint_bytes(dim: int, n: int, options: Options | None = None, nb: int = 1) -> int:
    """Device bytes of a problem (nb = 1) or a batch of nb problems; 0 if invalid."""
    o = options or default_options()
    return int(load_library().hh_footprint_batch_bytes(ctypes.byref(Grid(dim, n)), ctypes.byref(o), int(nb)))


def _ptr(t, numel=None):
    if t is None:
        return None
    if not t.is_cuda or not t.is_contiguous():
        raise ValueError("vectors must be contiguous CUDA tensors")
    if numel is not None and t.numel() != numel:
        raise ValueError(f"vector has {t.numel()} entries, expected {numel}")
    return ctypes.c_void_p(t.data_ptr())


def _prec_of(t):
    if t.dtype == torch.complex64:
        return HH_C64
    if t.dtype == torch.complex128:
        return HH_C128
    raise TypeError("vectors must be complex64 or complex128")


def _vec(v, nb):
    a = np.atleast_1d(np.asarray(v, dtype=np.float64))
    if a.size == 1 and nb > 1:
        a = np.full(nb, a[0])
    return a


class Problem:
    """A Helmholtz problem (scalar k, delta, delta_hat) or a batch of them (sequences of
    equal length): one grid, boundary tags and options, its own k/delta/delta_hat per
    problem.  Vectors of a batch hold the nb problems' level vectors one after another
    (flat, or shaped (nb, nodes)).  With options.formulation = HH_FORM_MIXED (one problem)
    the right side and solution of solve / precondition / apply_system hold the sigma
    entries and then the nodes (system_size() entries); level vectors stay nodal."""

    def __init__(self, dim, n, k, delta, delta_hat, bc, options: Options | None = None, stream=None):
        lib = load_library()
        batched = any(np.ndim(v) > 0 for v in (k, delta, delta_hat))
        nb = max(np.size(v) for v in (k, delta, delta_hat))
        ks, ds, dhs = (_vec(v, nb) for v in (k, delta, delta_hat))
        if not (ks.size == ds.size == dhs.size == nb):
            raise ValueError("k, delta and delta_hat need the same number of problems")
        self.dim, self.n, self.nb, self.batched = dim, n, int(nb), batched
        self.k = ks if batched else float(ks[0])
        self.options = options or default_options()
        bc = list(bc) + [0] * (6 - len(bc))
        arr = (ctypes.c_int * 6)(*bc)
        s = stream if stream is not None else torch.cuda.current_stream()
        self._stream = s
        handle = ctypes.c_void_p(s.cuda_stream)
        out = ctypes.c_void_p()
        dp = ctypes.POINTER(ctypes.c_double)
        self._keep = (np.ascontiguousarray(ks), np.ascontiguousarray(ds), np.ascontiguousarray(dhs))
        _check(lib.hh_create_batch(ctypes.byref(Grid(dim, n)), self.nb, *(a.ctypes.data_as(dp) for a in self._keep),
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

    def set_params(self, k, delta, delta_hat):
        """New k, delta, delta_hat for every problem (same grid and options); buffers kept."""
        ks, ds, dhs = (np.ascontiguousarray(_vec(v, self.nb)) for v in (k, delta, delta_hat))
        dp = ctypes.POINTER(ctypes.c_double)
        _check(self._lib.hh_set_params(self._p, ks.ctypes.data_as(dp), ds.ctypes.data_as(dp), dhs.ctypes.data_as(dp)))
        self.k = ks if self.batched else float(ks[0])

    def prepare(self):
        """Allocate the multigrid buffers and capture the preconditioner graph now."""
        _check(self._lib.hh_prepare(self._p))

    MODES = ("apply", "axpby", "jacobi", "hss_first", "jacobi2_zero", "prolong_jacobi", "resid_restrict",
             "prolong_jacobi2", "hss_first2", "jacobi2_zero_rr", "hss_first2_rr", "coarse")

    def autotune(self, precision=None):
        """Time the tile shapes of every stencil kernel and keep the fastest; returns
        {(level, mode): (rows, form)} for the tuned kernels."""
        prec = self.options.precision if precision is None else precision
        L = self.options.levels
        M = len(self.MODES)
        out = (ctypes.c_int * (L * M * 2))()
        _check(self._lib.hh_autotune(self._p, prec, out))
        return {(l, m): (out[(l * M + i) * 2], out[(l * M + i) * 2 + 1])
                for l in range(L) for i, m in enumerate(self.MODES) if out[(l * M + i) * 2]}

    def nodes(self, level=0) -> int:
        """Nodes of one problem's level-`level` vector."""
        return int(self._lib.hh_level_nodes(self._p, level))

    def size(self, level=0) -> int:
        """Entries of a batch vector of level `level` (nb x nodes)."""
        return self.nb * self.nodes(level)

    def system_size(self) -> int:
        """Entries of a batch right side / solution of hh_solve (nb x hh_vector_length):
        the nodes, or for a mixed problem its sigma entries and then the nodes."""
        return self.nb * int(self._lib.hh_vector_length(self._p))

    def apply_system(self, x, y=None):
        """y = the system operator x in FP64 (B_delta, or the mixed A_delta)."""
        y = torch.empty_like(x) if y is None else y
        n = self.system_size()
        _check(self._lib.hh_apply_system(self._p, _ptr(x, n), _ptr(y, n)))
        return y

    def zeros(self, level=0, dtype=torch.complex128):
        return torch.zeros(self.size(level), dtype=dtype, device="cuda")

    def _info(self, infos):
        return infos[0] if not self.batched else list(infos)

    # -- solver ------------------------------------------------------------
    def solve(self, rhs, tol=1e-8, x0=None, u=None):
        u = torch.empty_like(rhs) if u is None else u
        infos = (Info * self.nb)()
        n0 = self.system_size()
        st = self._lib.hh_solve(self._p, _ptr(rhs, n0), float(tol), _ptr(u, n0), _ptr(x0, n0), infos)
        _check(st, allow_not_converged=True)
        return u, self._info(infos)

    def solve_host(self, rhs: np.ndarray, tol=1e-8, out: np.ndarray | None = None, nodal=False):
        """Solve from host arrays (copies included); nodal=True: rhs is the nodal source f."""
        rhs = np.ascontiguousarray(rhs, dtype=np.complex128)
        out = np.empty_like(rhs) if out is None else out
        if rhs.size != self.system_size() or out.size != rhs.size or out.dtype != np.complex128 \
                or not out.flags.c_contiguous:
            raise ValueError("host vectors must be contiguous complex128 of nb x nodes entries")
        infos = (Info * self.nb)()
        fn = self._lib.hh_solve_host_nodal if nodal else self._lib.hh_solve_host
        st = fn(self._p, rhs.ctypes.data_as(ctypes.c_void_p), float(tol), out.ctypes.data_as(ctypes.c_void_p), infos)
        _check(st, allow_not_converged=True)
        return out, self._info(infos)

    # -- building blocks ------------------------------------------------------
    def apply(self, level, op, x, y=None):
        y = torch.empty_like(x) if y is None else y
        nl = self.size(level)
        _check(self._lib.hh_apply(self._p, level, OP[op], _prec_of(x), _ptr(x, nl), _ptr(y, nl)))
        return y

    def jacobi(self, level, b, x_in=None, x_out=None):
        x_out = torch.empty_like(b) if x_out is None else x_out
        nl = self.size(level)
        _check(self._lib.hh_jacobi(self._p, level, _prec_of(b), _ptr(b, nl), _ptr(x_in, nl), _ptr(x_out, nl)))
        return x_out

    def residual_restrict(self, level, b, x, rc=None):
        rc = torch.empty(self.size(level + 1), dtype=b.dtype, device=b.device) if rc is None else rc
        nl, nc = self.size(level), self.size(level + 1)
        _check(self._lib.hh_residual_restrict(self._p, level, _prec_of(b), _ptr(b, nl), _ptr(x, nl), _ptr(rc, nc)))
        return rc

    def prolong_correct(self, level, ec, x):
        nl, nc = self.size(level), self.size(level + 1)
        _check(self._lib.hh_prolong_correct(self._p, level, _prec_of(x), _ptr(ec, nc), _ptr(x, nl)))
        return x

    def vcycle(self, b, x=None):
        x = torch.empty_like(b) if x is None else x
        n0 = self.size(0)
        _check(self._lib.hh_vcycle(self._p, _prec_of(b), _ptr(b, n0), _ptr(x, n0)))
        return x

    def hss_rhs(self, u, r, rhs=None):
        rhs = torch.empty_like(r) if rhs is None else rhs
        n0 = self.size(0)
        _check(self._lib.hh_hss_rhs(self._p, _prec_of(r), _ptr(u, n0), _ptr(r, n0), _ptr(rhs, n0)))
        return rhs

    def precondition(self, r, z=None):
        z = torch.empty_like(r) if z is None else z
        n0 = self.system_size()
        _check(self._lib.hh_precondition(self._p, _ptr(r, n0), _ptr(z, n0)))
        return z

    def load_vector(self, f, b=None):
        b = torch.empty_like(f) if b is None else b
        n0 = self.size(0)
        _check(self._lib.hh_load_vector(self._p, _ptr(f, n0), _ptr(b, n0)))
        return b

    def dot(self, x, y):
        """x_b^H y_b per problem: a complex (single problem) or a list (batch)."""
        out = (ctypes.c_double * (2 * self.nb))()
        n0 = self.system_size()
        _check(self._lib.hh_dot(self._p, _ptr(x, n0), _ptr(y, n0), out))
        vals = [complex(out[2 * b], out[2 * b + 1]) for b in range(self.nb)]
        return vals if self.batched else vals[0]


class Pack:
    """Problems of different grids whose FGMRES solves share their preconditioner launches
    (hh_pack_*): add (problem, right side), run until members finish, take their results.
    Each result equals the member problem's own solve bit for bit."""

    def __init__(self, capacity=16):
        self._lib = load_library()
        self.capacity = int(capacity)
        out = ctypes.c_void_p()
        _check(self._lib.hh_pack_create(self.capacity, ctypes.byref(out)))
        self._k = out
        self._held = {}  # slot -> (problem, rhs, u) kept alive while the member runs

    def add(self, problem: "Problem", rhs, tol=1e-8, nodal=False) -> int:
        """Add a member: rhs a CUDA complex128 load vector (u returned on the device), or a host
        numpy array (load vector, or with nodal=True the nodal source f); returns its slot."""
        slot = ctypes.c_int()
        if isinstance(rhs, np.ndarray):
            rhs = np.ascontiguousarray(rhs, dtype=np.complex128)
            u = np.empty_like(rhs)
            io, rp, up = (2 if nodal else 1), rhs.ctypes.data_as(ctypes.c_void_p), u.ctypes.data_as(ctypes.c_void_p)
            if rhs.size != problem.system_size():
                raise ValueError("right side has the wrong size")
        else:
            u = torch.empty_like(rhs)
            io, rp, up = 0, _ptr(rhs, problem.system_size()), _ptr(u, problem.system_size())
        _check(self._lib.hh_pack_add(self._k, problem._p, rp, io, float(tol), up, ctypes.byref(slot)))
        self._held[slot.value] = (problem, rhs, u)
        return slot.value

    def run(self, max_rounds=0):
        """Run until at least one member finishes (or max_rounds rounds, if > 0); returns the
        finished slots."""
        done = (ctypes.c_int * self.capacity)()
        nd = ctypes.c_int()
        _check(self._lib.hh_pack_run(self._k, int(max_rounds), done, ctypes.byref(nd)))
        return [done[i] for i in range(nd.value)]

    def take(self, slot):
        """(u, info) of a finished member; frees its slot."""
        info = Info()
        st = self._lib.hh_pack_take(self._k, int(slot), ctypes.byref(info))
        _, _, u = self._held.pop(slot, (None, None, None))
        _check(st, allow_not_converged=True)
        return u, info

    def members(self) -> int:
        return int(self._lib.hh_pack_members(self._k))

    def close(self):
        if getattr(self, "_k", None):
            self._lib.hh_pack_destroy(self._k)
            self._k = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


class Server:
    """Continuous-batching solve server (hh_server_*): submit host right sides of any grid
    and wavenumber, wait for the solutions.  Solves run concurrently on the device, admitted
    as worker slots and the device budget allow."""

    def __init__(self, slots=4, budget_bytes=8 << 30, options: Options | None = None):
        self._lib = load_library()
        self.options = options or default_options()
        out = ctypes.c_void_p()
        _check(self._lib.hh_server_create(int(slots), int(budget_bytes), ctypes.byref(self.options),
                                          ctypes.byref(out)))
        self._s = out
        self._pending = {}

    def submit(self, dim, n, k, delta, delta_hat, bc, rhs: np.ndarray, tol=1e-8, nodal=False) -> int:
        """Queue a solve of B u = rhs (complex128 load vector, or with nodal=True the nodal
        source f and b = M f; (n+1)^dim entries); returns a ticket."""
        rhs = np.ascontiguousarray(rhs, dtype=np.complex128)
        if rhs.size != (n + 1) ** dim:
            raise ValueError("right side has the wrong number of entries")
        u = np.empty_like(rhs)
        bcs = list(bc) + [0] * (6 - len(bc))
        req = Request(Grid(dim, n), float(k), float(delta), float(delta_hat), (ctypes.c_int * 6)(*bcs), float(tol),
                      1 if nodal else 0)
        t = ctypes.c_longlong()
        _check(self._lib.hh_server_submit(self._s, ctypes.byref(req), rhs.ctypes.data_as(ctypes.c_void_p),
                                          u.ctypes.data_as(ctypes.c_void_p), ctypes.byref(t)))
        self._pending[t.value] = (rhs, u)  # keep the host arrays alive until waited for
        return t.value

    def wait(self, ticket):
        """(u, info, latency_s, queue_s) of a submitted request."""
        info = Info()
        lat, qs = ctypes.c_double(), ctypes.c_double()
        st = self._lib.hh_server_wait(self._s, ticket, ctypes.byref(info), ctypes.byref(lat), ctypes.byref(qs))
        _, u = self._pending.pop(ticket, (None, None))
        _check(st, allow_not_converged=True)
        return u, info, lat.value, qs.value

    def set_fallback(self, options: Options | None, delta_hat: float = 2.0):
        """Solve requests that do not converge once more with these options and delta_hat
        (None removes the fallback); see hh_server_set_fallback."""
        self._fallback = options  # kept alive: the server copies it, the binding keeps the original
        _check(self._lib.hh_server_set_fallback(self._s, ctypes.byref(options) if options is not None else None,
                                                float(delta_hat)))

    def set_pack(self, capacity=16, max_hss_steps=0):
        """Run the server's 2D requests with at most max_hss_steps HSS steps (0: all) as members
        of one pack (hh_server_set_pack)."""
        _check(self._lib.hh_server_set_pack(self._s, int(capacity), int(max_hss_steps)))

    def stats(self) -> dict:
        out = ServerStats()
        _check(self._lib.hh_server_get_stats(self._s, ctypes.byref(out)))
        return out.as_dict()

    def close(self):
        if getattr(self, "_s", None):
            self._lib.hh_server_destroy(self._s)
            self._s = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()
