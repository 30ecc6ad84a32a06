"""FP64 CPU oracle for the mixed formulation of the Helmholtz problem.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import this module: only
``tests/``, ``__graft_entry__.smoke()`` and the CPU legs of ``bench.py`` use it.  It shares
no code with the CUDA library.

What it computes (Cotter, Hope-Collins & Knook, arXiv 2506.18694):

* the mixed system of Sec. 2 (Eq. "mixed"): (sigma, u) in V_h x Q_h with
      (delta - i k) <sigma, tau> - <grad u, tau> = 0                     for all tau,
      <sigma, grad v> + (delta - i k) <u, v> + <<u, v>> = <f, v> / (delta - i k)  for all v,
  where <<.,.>> is the boundary mass on the Sommerfeld sides;
* the gamma = k HSS iteration of Def. 3.5 / Eq. HSSm, (k H + S) U' = c1 (k H - S) U + c2 F,
  with H = delta Ms (+) (delta M + M_Gamma) and S the skew part, and the shifted-HSS
  preconditioner of Def. 4.2 (the same iteration with delta replaced by delta_hat, from
  U_0 = 0, ceil(k^theta) steps), both solved directly as 2 x 2 block systems and through the
  elimination of sigma that the embedding property allows (Sec. 3.2): the u-equation becomes
      A_mix u' = K u' + k^2 (dh - i)^2 M u' + k^2 (dh - i) M_Gamma u' = right side,
  a primal-type shifted operator, solved by LU or by the primal oracle's multigrid cycles;
* flexible GMRES (the primal oracle's) on the mixed system with that preconditioner.

Spaces.  Q_h is Q1 (as in the primal oracle).  The paper's V_h = (DG_{p-1})^d on triangles
contains grad Q_h; on quadrilaterals (DQ0)^d does not.  Here V_h is the smallest broken
space that does: on each cell the a-th component is multilinear in the coordinates other
than a and constant along a (2D: sigma_x in span{1, y}, sigma_y in span{1, x}), with the
tensor products of the 1D hat functions of the other axes as its basis.  sigma DoFs are
numbered (cell, component a, local vertex s of the other axes), cells x fastest.

Every function here is pinned in ``tests/test_oracle_mixed_pins.py``.
"""
from __future__ import annotations

import math

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from oracle import hh_oracle as O


def _other_axes(dim, a):
    return [b for b in range(dim) if b != a]


def _psi(s, a, xi, dim):
    """Basis function s of component a of V_h at reference point xi of [0,1]^dim."""
    v = 1.0
    for bit, b in enumerate(_other_axes(dim, a)):
        x = xi[b]
        v *= x if (s >> bit) & 1 else (1.0 - x)
    return v


def sigma_element(dim, h):
    """Cell matrices by tensor Gauss quadrature (2 points per axis, exact here):
    Ms_e[a][s, t] = int psi_{a,s} psi_{a,t} and G_e[a][s, A] = int psi_{a,s} d phi_A / dx_a."""
    ns = 2 ** (dim - 1)
    nodes = O._local_nodes(dim)
    Ms = np.zeros((dim, ns, ns))
    Ge = np.zeros((dim, ns, len(nodes)))
    for q in np.ndindex(*([2] * dim)):
        xi = [O._G1[qi] for qi in q]
        w = np.prod([O._W1[qi] for qi in q]) * h ** dim
        for a in range(dim):
            for s in range(ns):
                ps = _psi(s, a, xi, dim)
                for t in range(ns):
                    Ms[a, s, t] += w * ps * _psi(t, a, xi, dim)
                for A, an in enumerate(nodes):
                    Ge[a, s, A] += w * ps * O._dphi(an, xi, a) / h
    return Ms, Ge


def assemble_mixed(grid):
    """(Ms, G): the V_h mass matrix (block diagonal by cell) and the coupling
    G[(cell, a, s), node] = int psi_{a,s} d phi_node / dx_a, columns of Dirichlet nodes zero."""
    dim = grid.dim
    ns = 2 ** (dim - 1)
    cells, g = O._cell_vertex_globals(grid)
    nc = cells.shape[0]
    nsig = nc * dim * ns
    Mse, Ge = sigma_element(dim, grid.h)
    rows, cols, vals = [], [], []
    grow, gcol, gval = [], [], []
    for a in range(dim):
        for s in range(ns):
            r = np.arange(nc) * dim * ns + a * ns + s
            for t in range(ns):
                rows.append(r)
                cols.append(np.arange(nc) * dim * ns + a * ns + t)
                vals.append(np.full(nc, Mse[a, s, t]))
            for A in range(2 ** dim):
                grow.append(r)
                gcol.append(g[:, A])
                gval.append(np.full(nc, Ge[a, s, A]))
    Ms = sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))), shape=(nsig, nsig))
    G = sp.csr_matrix((np.concatenate(gval), (np.concatenate(grow), np.concatenate(gcol))), shape=(nsig, grid.N))
    G = (G @ sp.diags(grid.free().astype(float))).tocsr()
    G.eliminate_zeros()
    return Ms, G


def coeff_mix(k, dh):
    """The u-operator after eliminating sigma from Def. 4.2: K + k^2 (dh - i)^2 M + k^2 (dh - i) M_Gamma."""
    s = dh - 1j
    return (1.0 + 0j, k * k * s * s, k * k * s)


class MixedProblem:
    """A mixed-formulation problem: grid, k, delta (the system), delta_hat (the preconditioner),
    multigrid options for the eliminated u-equation."""

    def __init__(self, grid, k, delta, delta_hat, opts=None):
        if k <= 0 or delta < 0 or delta_hat <= 0:
            raise ValueError("need k > 0, delta >= 0, delta_hat > 0")
        self.grid, self.k, self.delta, self.delta_hat = grid, k, delta, delta_hat
        self.K, self.M, self.MG = O.assemble(grid)
        self.Ms, self.G = assemble_mixed(grid)
        self.ns = self.Ms.shape[0]
        self.N = grid.N
        self.free_u = grid.free()
        self.free = np.concatenate([np.ones(self.ns, dtype=bool), self.free_u])
        self.Amix = O.combine((self.K, self.M, self.MG), coeff_mix(k, delta_hat))
        self.opts = opts or O.Options()
        self._mg = None
        self._lu = {}

    # -- block operators ---------------------------------------------------------------
    def block(self, cs, cu, cg, sign_g):
        """[[cs Ms, -sign_g G], [sign_g G^T, cu M + cg M_Gamma]] on (sigma, u)."""
        return sp.bmat([[cs * self.Ms, -sign_g * self.G],
                        [sign_g * self.G.T, cu * self.M + cg * self.MG]]).tocsr()

    def A(self, delta=None):
        """The mixed system operator A_delta (Sec. 2, Eq. mixed); delta defaults to the problem's."""
        d = self.delta if delta is None else delta
        z = d - 1j * self.k
        return self.block(z, z, 1.0, 1.0)

    def H(self, dh):
        """Gram matrix of the H_mixed inner product with delta -> dh (Sec. 3.2)."""
        return self.block(dh, dh, 1.0, 0.0).real

    def rhs(self, f_nodal, delta=None):
        """(F_sigma, F_u) = (0, M f / (delta - i k)) for a nodal source f."""
        d = self.delta if delta is None else delta
        bu = (self.M @ f_nodal) / (d - 1j * self.k)
        return np.concatenate([np.zeros(self.ns, dtype=complex), bu])

    def split(self, U):
        return U[: self.ns], U[self.ns:]

    def _solve_free(self, key, A, b):
        f = np.nonzero(self.free)[0]
        if key not in self._lu:
            self._lu[key] = spla.splu(A[f][:, f].tocsc())
        x = np.zeros(A.shape[0], dtype=complex)
        x[f] = self._lu[key].solve(np.asarray(b, dtype=complex)[f])
        return x

    def lu_solve(self, b, delta=None):
        """Direct solution of A_delta U = b (free DoFs)."""
        d = self.delta if delta is None else delta
        return self._solve_free(("A", d), self.A(d), b)

    # -- HSS (Def. 3.5 with gamma = k; Def. 4.2 with delta -> delta_hat) ------------------
    def hss_lhs(self, dh):
        k = self.k
        return self.block(k * (dh - 1j), k * (dh - 1j), k, 1.0)

    def hss_rhs_op(self, dh):
        k = self.k
        return self.block(k * (dh + 1j), k * (dh + 1j), k, -1.0)

    def hss_step_direct(self, U, R, dh=None):
        """One HSS step solved as the 2 x 2 block system of Def. 4.2."""
        dh = self.delta_hat if dh is None else dh
        c1, c2 = O.hss_weights(self.k)
        b = c1 * (self.hss_rhs_op(dh) @ U) + c2 * R
        return self._solve_free(("hss", dh), self.hss_lhs(dh), b)

    def hss_step_eliminated(self, U, R, inner=None):
        """The same step through the elimination of sigma (Sec. 3.2): the tau-rows give
        sigma' = Ms^{-1} (g_s + G u') / (k (dh - i)); substituting into the v-rows and
        multiplying by k (dh - i) leaves A_mix u' = k (dh - i) g_u - G^T Ms^{-1} g_s, with
        g_s, g_u the right sides of the tau- and v-rows.  ``inner`` solves A_mix (default LU)."""
        k, dh = self.k, self.delta_hat
        c1, c2 = O.hss_weights(k)
        sig, u = self.split(U)
        Rs, Ru = self.split(R)
        g_s = c1 * (k * (dh + 1j) * (self.Ms @ sig) + self.G @ u) + c2 * Rs
        g_u = c1 * (k * (dh + 1j) * (self.M @ u) - self.G.T @ sig + k * (self.MG @ u)) + c2 * Ru
        ms_inv_gs = self.ms_solve(g_s)
        rhs_u = k * (dh - 1j) * g_u - self.G.T @ ms_inv_gs
        rhs_u = rhs_u * self.free_u
        u_new = self.amix_lu(rhs_u) if inner is None else inner(rhs_u)
        sig_new = self.ms_solve(g_s + self.G @ u_new) / (k * (dh - 1j))
        return np.concatenate([sig_new, u_new])

    def ms_solve(self, g):
        if "Ms" not in self._lu:
            self._lu["Ms"] = spla.splu(self.Ms.tocsc())
        g = np.asarray(g, dtype=complex)
        lu = self._lu["Ms"]
        return lu.solve(np.ascontiguousarray(g.real)) + 1j * lu.solve(np.ascontiguousarray(g.imag))

    def amix_lu(self, b):
        f = np.nonzero(self.free_u)[0]
        if "Amix" not in self._lu:
            self._lu["Amix"] = spla.splu(self.Amix[f][:, f].tocsc())
        x = np.zeros(self.N, dtype=complex)
        x[f] = self._lu["Amix"].solve(np.asarray(b, dtype=complex)[f])
        return x

    def mg(self):
        """The primal oracle's multigrid hierarchy, built for A_mix instead of A_L."""
        if self._mg is None:
            self._mg = O.Problem(self.grid, self.k, self.delta, self.delta_hat, self.opts,
                                 al_coeff=coeff_mix(self.k, self.delta_hat))
        return self._mg

    def prec(self, R, inner="mg"):
        """Shifted-HSS preconditioner of Def. 4.2: U_0 = 0, ceil(k^theta) eliminated steps,
        the u-equation solved by multigrid cycles (``inner="mg"``) or LU (``inner=None``)."""
        solve = self.mg().mg_solve if inner == "mg" else inner
        U = np.zeros(self.ns + self.N, dtype=complex)
        for _ in range(O.n_hss(self.k, self.opts.theta)):
            U = self.hss_step_eliminated(U, R, solve)
        return U

    def solve(self, b, tol, inner="mg", restart=30, max_it=300):
        """FGMRES on A_delta U = b preconditioned by Def. 4.2 (the primal oracle's FGMRES)."""
        A = self.A()
        return O.fgmres(lambda x: A @ x, b, lambda r: self.prec(r, inner), tol, restart=restart, max_it=max_it)
