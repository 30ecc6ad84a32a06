"""ctypes binding of the plain-C OpenMP oracle (oracle/hss_omp.c).

TEST INFRASTRUCTURE ONLY: used by tests/, by __graft_entry__.build() (which compiles it)
and by the CPU legs of bench.py.  The CUDA product never imports it.

The C code restates the Python oracle's V-cycle, shifted-HSS preconditioner (Def. 4.1)
and flexible GMRES (Sec. 5.1) for grids of millions of nodes; the CSR matrices it runs on
are the ones hh_oracle.Problem assembles, handed over without copies.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np
import scipy.sparse as sp

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "hss_omp.c")
LIB = os.path.join(HERE, "libhss_omp.so")
MAX_LEVELS = 12

_lib = None


def build(force: bool = False) -> str:
    """Compile hss_omp.c with gcc and OpenMP into oracle/libhss_omp.so (if stale)."""
    if force or not os.path.exists(LIB) or os.path.getmtime(LIB) < os.path.getmtime(SRC):
        tmp = LIB + ".tmp"
        subprocess.run(["gcc", "-std=c11", "-O2", "-fopenmp", "-fPIC", "-shared", "-o", tmp, SRC, "-lm"],
                       check=True)
        os.replace(tmp, LIB)
    return LIB


class _CSR(ctypes.Structure):
    _fields_ = [("nrows", ctypes.c_longlong), ("rowptr", ctypes.c_void_p), ("col", ctypes.c_void_p),
                ("val", ctypes.c_void_p), ("rval", ctypes.c_void_p)]


class _Problem(ctypes.Structure):
    _fields_ = [("levels", ctypes.c_int), ("N", ctypes.c_longlong * MAX_LEVELS),
                ("AL", _CSR * MAX_LEVELS), ("dinv", ctypes.c_void_p * MAX_LEVELS),
                ("P", _CSR * MAX_LEVELS), ("PT", _CSR * MAX_LEVELS), ("AR", _CSR), ("B", _CSR),
                ("k", ctypes.c_double), ("omega", ctypes.c_double), ("nu_pre", ctypes.c_int),
                ("nu_post", ctypes.c_int), ("nu_coarse", ctypes.c_int), ("cycles_per_hss", ctypes.c_int),
                ("nhss", ctypes.c_int)]


def load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        P = ctypes.c_void_p
        lib.hss_set_threads.argtypes = [ctypes.c_int]
        lib.hss_set_threads.restype = None
        lib.hss_max_threads.argtypes = []
        lib.hss_max_threads.restype = ctypes.c_int
        lib.hss_vcycle.argtypes = [P, ctypes.c_int, P, P]
        lib.hss_vcycle.restype = ctypes.c_int
        lib.hss_mg_solve.argtypes = [P, P, P]
        lib.hss_mg_solve.restype = ctypes.c_int
        lib.hss_prec.argtypes = [P, P, P]
        lib.hss_prec.restype = ctypes.c_int
        lib.hss_time_steps.argtypes = [P, P, ctypes.c_double, ctypes.c_longlong, ctypes.POINTER(ctypes.c_double)]
        lib.hss_time_steps.restype = ctypes.c_longlong
        lib.hss_fgmres.argtypes = [P, P, ctypes.c_double, ctypes.c_int, ctypes.c_int, P,
                                   ctypes.POINTER(ctypes.c_double)]
        lib.hss_fgmres.restype = ctypes.c_int
        _lib = lib
    return _lib


def _ptr(a):
    return ctypes.c_void_p(a.ctypes.data)


class COracle:
    """The C oracle over the matrices of an hh_oracle.Problem (V-cycles with Jacobi only)."""

    def __init__(self, prob):
        from oracle import hh_oracle as O

        o = prob.opts
        if o.gamma != 1 or o.smoother != "jacobi":
            raise ValueError("the C oracle runs V-cycles with the Jacobi smoother")
        L = len(prob.AL)
        if L > MAX_LEVELS:
            raise ValueError("too many levels")
        self.N = prob.grid.N
        self._keep = []  # arrays the C side points into
        st = _Problem()
        st.levels = L
        for l in range(L):
            st.N[l] = prob.grids[l].N
            st.AL[l] = self._csr(prob.AL[l], complex)
            st.dinv[l] = self._arr(np.asarray(prob.Dinv[l], dtype=complex)).value
            if l + 1 < L:
                st.P[l] = self._csr(prob.P[l], float)
                st.PT[l] = self._csr(prob.P[l].T.tocsr(), float)
        st.AR = self._csr(prob.AR0, complex)
        st.B = self._csr(prob.B, complex)
        st.k = prob.k
        st.omega = o.omega
        st.nu_pre, st.nu_post, st.nu_coarse = o.nu_pre, o.nu_post, o.nu_coarse
        st.cycles_per_hss = o.cycles_per_hss
        st.nhss = O.n_hss(prob.k, o.theta)
        self._st = st
        self._lib = load()

    def _arr(self, a):
        a = np.ascontiguousarray(a)
        self._keep.append(a)
        return ctypes.c_void_p(a.ctypes.data)

    def _csr(self, A, kind):
        A = sp.csr_matrix(A)
        c = _CSR()
        c.nrows = A.shape[0]
        c.rowptr = self._arr(A.indptr.astype(np.int64)).value
        c.col = self._arr(A.indices.astype(np.int32)).value
        if kind is complex:
            c.val = self._arr(A.data.astype(complex)).value
            c.rval = None
        else:
            c.val = None
            c.rval = self._arr(A.data.astype(float)).value
        return c

    @property
    def _p(self):
        return ctypes.byref(self._st)

    @staticmethod
    def threads(t=None):
        lib = load()
        if t:
            lib.hss_set_threads(int(t))
        return lib.hss_max_threads()

    def _vec(self, v, n):
        v = np.ascontiguousarray(v, dtype=complex)
        if v.shape != (n,):
            raise ValueError("wrong vector size")
        return v

    def vcycle(self, l, b):
        b = self._vec(b, self._st.N[l])
        x = np.empty_like(b)
        if self._lib.hss_vcycle(self._p, l, _ptr(b), _ptr(x)):
            raise MemoryError("hss_vcycle")
        return x

    def mg_solve(self, b):
        b = self._vec(b, self.N)
        x = np.empty_like(b)
        if self._lib.hss_mg_solve(self._p, _ptr(b), _ptr(x)):
            raise MemoryError("hss_mg_solve")
        return x

    def prec(self, r):
        r = self._vec(r, self.N)
        z = np.empty_like(r)
        if self._lib.hss_prec(self._p, _ptr(r), _ptr(z)):
            raise MemoryError("hss_prec")
        return z

    def time_steps(self, r, seconds, max_steps=1 << 40):
        """HSS steps from u = 0 for about `seconds`: (steps, wall seconds)."""
        r = self._vec(r, self.N)
        el = ctypes.c_double(0.0)
        steps = self._lib.hss_time_steps(self._p, _ptr(r), float(seconds), int(max_steps), ctypes.byref(el))
        if steps < 0:
            raise MemoryError("hss_time_steps")
        return int(steps), el.value

    def fgmres(self, b, tol, restart=30, max_it=1000, x0=None):
        """FGMRES on B x = b with the shifted-HSS preconditioner: (x, iterations, rel. residual)."""
        b = self._vec(b, self.N)
        x = np.zeros_like(b) if x0 is None else self._vec(x0, self.N).copy()
        rr = ctypes.c_double(0.0)
        its = self._lib.hss_fgmres(self._p, _ptr(b), float(tol), int(restart), int(max_it), _ptr(x),
                                   ctypes.byref(rr))
        if its < 0:
            raise MemoryError("hss_fgmres")
        return x, its, rr.value
