"""FP64 CPU oracle for the shifted-HSS Helmholtz solver.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import this module:
only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline / reference
legs of ``bench.py`` use it.  It shares no code with the CUDA library.

What it computes (Cotter, Hope-Collins & Knook, "Shifted HSS solvers for the
indefinite Helmholtz equation", arXiv 2506.18694):

* the primal weak form b_delta of Sec. 2 (the bilinear form of Eq. "primal H1")
  discretised with Q1 elements on a uniform grid of the unit square / cube:
  every matrix is assembled element by element in CSR from Gauss quadrature of
  the bilinear / trilinear basis (no Kronecker shortcut, so the Kronecker form
  can serve as an independent check);
* the gamma = k HSS iteration of Def. 3.1 (Eq. "primal-hss-system") and the
  shifted-HSS preconditioner of Def. 4.1 (Eq. "HSSpc primal"), whose inner
  systems are approximated here by a multigrid V- or W-cycle with scaled Jacobi
  smoothing, or GMRES with a Jacobi preconditioner as the smoother (Sec. 5.3),
  prolongation by bi/trilinear interpolation and restriction R = P^T;
* flexible GMRES (Saad 1993, used as the outer method in Sec. 5.1) with right
  preconditioning, modified Gram-Schmidt and Givens rotations;
* a direct sparse LU solve of the same discrete system, which is the exact
  answer every iterative result is measured against.

All arithmetic is complex128 / float64.  Vectors are full-length over the
(n+1)^d grid nodes, lexicographic with x fastest; entries at Dirichlet nodes
are held at zero.

Parity status: every function here is pinned by a test in
``tests/test_oracle_pins.py`` (closed forms, identities, brute force, LU).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

SOMMERFELD = 0  # boundary part Gamma: du/dn - (-delta + i k) u = 0   (Sec. 1)
DIRICHLET = 1   # boundary part dOmega_0: u = 0                         (Sec. 1)


# ---------------------------------------------------------------------------
# Grid
# ---------------------------------------------------------------------------
@dataclass
class Grid:
    """Uniform grid of the unit square (dim=2) or cube (dim=3) with n cells per axis.

    ``bc`` lists the tag of each side in the order -x, +x, -y, +y, -z, +z.
    """

    dim: int
    n: int
    bc: tuple

    def __post_init__(self):
        if self.dim not in (2, 3):
            raise ValueError("dim must be 2 or 3")
        self.bc = tuple(int(t) for t in self.bc[: 2 * self.dim])
        self.h = 1.0 / self.n
        self.nn = self.n + 1
        self.N = self.nn ** self.dim

    def index(self, *ijk):
        """Global node number of integer node coordinates (x fastest)."""
        g = 0
        stride = 1
        for c in ijk:
            g = g + stride * np.asarray(c)
            stride *= self.nn
        return g

    def node_ijk(self):
        """Integer coordinates of every node, shape (N, dim)."""
        axes = [np.arange(self.nn)] * self.dim
        mesh = np.meshgrid(*axes[::-1], indexing="ij")  # slowest axis first
        cols = [m.ravel() for m in mesh[::-1]]            # back to (x, y, z)
        return np.stack(cols, axis=1)

    def coords(self):
        return self.node_ijk() * self.h

    def dirichlet_nodes(self):
        """Boolean mask of the nodes on a Dirichlet-tagged side."""
        ijk = self.node_ijk()
        mask = np.zeros(self.N, dtype=bool)
        for ax in range(self.dim):
            if self.bc[2 * ax] == DIRICHLET:
                mask |= ijk[:, ax] == 0
            if self.bc[2 * ax + 1] == DIRICHLET:
                mask |= ijk[:, ax] == self.n
        return mask

    def free(self):
        return ~self.dirichlet_nodes()

    def coarse(self):
        if self.n % 2:
            raise ValueError("cannot coarsen an odd grid")
        return Grid(self.dim, self.n // 2, self.bc)


# ---------------------------------------------------------------------------
# Element matrices by Gauss quadrature of the Q1 basis (exact for Q1 products)
# ---------------------------------------------------------------------------
_G1 = np.array([0.5 - 0.5 / math.sqrt(3.0), 0.5 + 0.5 / math.sqrt(3.0)])  # 2-pt Gauss on [0,1]
_W1 = np.array([0.5, 0.5])


def _local_nodes(dim):
    """Local vertex multi-indices a in {0,1}^dim, local number = a_x + 2 a_y + 4 a_z."""
    return [tuple((a >> s) & 1 for s in range(dim)) for a in range(2 ** dim)]


def _phi(a, xi):
    """Reference Q1 basis function for vertex a at reference point xi in [0,1]^dim."""
    v = 1.0
    for ad, x in zip(a, xi):
        v *= x if ad else (1.0 - x)
    return v


def _dphi(a, xi, axis):
    """d phi_a / d xi_axis on the reference cell."""
    v = 1.0
    for d, (ad, x) in enumerate(zip(a, xi)):
        if d == axis:
            v *= 1.0 if ad else -1.0
        else:
            v *= x if ad else (1.0 - x)
    return v


def element_matrices(dim, h):
    """Cell stiffness K^e[a,b] = int grad phi_a . grad phi_b and mass M^e[a,b] = int phi_a phi_b.

    Tensor Gauss quadrature with 2 points per axis on a cell of side h.  These are
    the volume terms of the primal bilinear form b_delta (Sec. 2).
    """
    nodes = _local_nodes(dim)
    nl = len(nodes)
    Ke = np.zeros((nl, nl))
    Me = np.zeros((nl, nl))
    for q in np.ndindex(*([2] * dim)):
        xi = [_G1[qi] for qi in q]
        w = np.prod([_W1[qi] for qi in q]) * h ** dim
        for A, a in enumerate(nodes):
            for B, b in enumerate(nodes):
                Me[A, B] += w * _phi(a, xi) * _phi(b, xi)
                g = 0.0
                for ax in range(dim):
                    g += _dphi(a, xi, ax) * _dphi(b, xi, ax) / (h * h)
                Ke[A, B] += w * g
    return Ke, Me


def face_mass_matrix(dim, h, axis, side):
    """Boundary mass int_face phi_a phi_b dS on the cell face {xi_axis = side}.

    Returned over all 2^dim local vertices (rows/cols of vertices off the face are
    zero).  This is the boundary term of b_delta (Sec. 2).
    """
    nodes = _local_nodes(dim)
    nl = len(nodes)
    Fe = np.zeros((nl, nl))
    others = [ax for ax in range(dim) if ax != axis]
    for q in np.ndindex(*([2] * (dim - 1))):
        xi = [0.0] * dim
        xi[axis] = float(side)
        for o, qi in zip(others, q):
            xi[o] = _G1[qi]
        w = np.prod([_W1[qi] for qi in q]) * h ** (dim - 1)
        for A, a in enumerate(nodes):
            for B, b in enumerate(nodes):
                Fe[A, B] += w * _phi(a, xi) * _phi(b, xi)
    return Fe


# ---------------------------------------------------------------------------
# Global assembly (element loop, vectorised over cells) with Dirichlet masking
# ---------------------------------------------------------------------------
def _cell_vertex_globals(grid):
    """(ncells, 2^dim) array: global node number of each local vertex of each cell."""
    n, dim = grid.n, grid.dim
    cells = np.stack(np.meshgrid(*([np.arange(n)] * dim)[::-1], indexing="ij")[::-1], axis=-1)
    cells = cells.reshape(-1, dim)  # (ncells, dim) integer cell origins, x fastest
    out = np.zeros((cells.shape[0], 2 ** dim), dtype=np.int64)
    for A, a in enumerate(_local_nodes(dim)):
        out[:, A] = grid.index(*[cells[:, d] + a[d] for d in range(dim)])
    return cells, out


def _scatter(rows_of_cells, Ee, N):
    nl = Ee.shape[0]
    r = np.repeat(rows_of_cells, nl, axis=1).ravel()
    c = np.tile(rows_of_cells, (1, nl)).ravel()
    v = np.tile(Ee.ravel(), rows_of_cells.shape[0])
    return sp.csr_matrix((v, (r, c)), shape=(N, N))


def _mask(grid, A):
    f = sp.diags(grid.free().astype(float))
    out = (f @ A @ f).tocsr()
    out.eliminate_zeros()
    return out


def assemble(grid):
    """Return the masked real CSR matrices (K, M, M_Gamma) of the primal form (Sec. 2).

    K: stiffness, M: mass, M_Gamma: boundary mass over the Sommerfeld-tagged sides.
    Rows and columns of Dirichlet nodes are zero (those unknowns are eliminated).
    """
    dim, N = grid.dim, grid.N
    Ke, Me = element_matrices(dim, grid.h)
    cells, g = _cell_vertex_globals(grid)
    K = _scatter(g, Ke, N)
    M = _scatter(g, Me, N)
    MG = sp.csr_matrix((N, N))
    for axis in range(dim):
        for side in (0, 1):
            if grid.bc[2 * axis + side] != SOMMERFELD:
                continue
            on = cells[:, axis] == (0 if side == 0 else grid.n - 1)
            Fe = face_mass_matrix(dim, grid.h, axis, side)
            MG = MG + _scatter(g[on], Fe, N)
    return _mask(grid, K), _mask(grid, M), _mask(grid, MG.tocsr())


def apply_elementwise(grid, coeff, x):
    """(c_K K + c_M M + c_G M_Gamma) x without assembling: sum over cells of the element
    matrices times the cell's nodal values, plus the Sommerfeld face terms; rows and
    columns of Dirichlet nodes masked.  Same operator as ``combine(assemble(grid), coeff)``,
    for grids too large to assemble (millions of nodes)."""
    dim, N = grid.dim, grid.N
    cK, cM, cG = coeff
    Ke, Me = element_matrices(dim, grid.h)
    Ae = cK * Ke + cM * Me
    free = grid.free()
    xm = np.where(free, np.asarray(x, dtype=complex), 0.0)
    cells, g = _cell_vertex_globals(grid)
    y = np.zeros(N, dtype=complex)
    xe = xm[g]                       # (ncells, 2^dim)
    ye = xe @ Ae.T                   # element contributions
    for A in range(g.shape[1]):
        y += np.bincount(g[:, A], weights=ye[:, A].real, minlength=N) + \
            1j * np.bincount(g[:, A], weights=ye[:, A].imag, minlength=N)
    for axis in range(dim):
        for side in (0, 1):
            if grid.bc[2 * axis + side] != SOMMERFELD:
                continue
            on = cells[:, axis] == (0 if side == 0 else grid.n - 1)
            Fe = cG * face_mass_matrix(dim, grid.h, axis, side)
            gf = g[on]
            yf = xm[gf] @ Fe.T
            for A in range(gf.shape[1]):
                y += np.bincount(gf[:, A], weights=yf[:, A].real, minlength=N) + \
                    1j * np.bincount(gf[:, A], weights=yf[:, A].imag, minlength=N)
    return np.where(free, y, 0.0)


def diag_elementwise(grid, coeff):
    """diag(c_K K + c_M M + c_G M_Gamma) from the element and face matrices' diagonals (no
    assembly); zero at Dirichlet nodes."""
    dim, N = grid.dim, grid.N
    cK, cM, cG = coeff
    Ke, Me = element_matrices(dim, grid.h)
    de = np.diag(cK * Ke + cM * Me)
    cells, g = _cell_vertex_globals(grid)
    d = np.zeros(N, dtype=complex)
    for A in range(g.shape[1]):
        d += np.bincount(g[:, A], minlength=N) * de[A]
    for axis in range(dim):
        for side in (0, 1):
            if grid.bc[2 * axis + side] != SOMMERFELD:
                continue
            on = cells[:, axis] == (0 if side == 0 else grid.n - 1)
            df = cG * np.diag(face_mass_matrix(dim, grid.h, axis, side))
            for A in range(g.shape[1]):
                d += np.bincount(g[on][:, A], minlength=N) * df[A]
    return np.where(grid.free(), d, 0.0)


# ---------------------------------------------------------------------------
# Operator coefficient triples (c_K, c_M, c_Gamma): op = c_K K + c_M M + c_Gamma M_Gamma
# ---------------------------------------------------------------------------
def coeff_B(k, delta):
    """B_delta of b_delta (Sec. 2): K + (-delta + i k)^2 M - (-delta + i k) M_Gamma."""
    s = -delta + 1j * k
    return (1.0 + 0j, s * s, -s)


def coeff_AL(k, dh):
    """Left operator of Def. 4.1 (Eq. HSSpc primal), delta replaced by delta_hat."""
    return (1.0 + 0j, dh * dh - k * k - 2j * dh * k * k, dh - 1j * k * k)


def coeff_AR(k, dh):
    """Right operator of Def. 4.1 (Eq. HSSpc primal), without the factor (k-1)/(k+1)."""
    return (-1.0 + 0j, k * k - dh * dh - 2j * dh * k * k, -dh - 1j * k * k)


def coeff_H(k, dh):
    """Inner-product matrix H = 2 delta k M + k M_Gamma of Sec. 3.1 (delta -> delta_hat)."""
    return (0.0 + 0j, 2.0 * dh * k + 0j, k + 0j)


def hss_weights(k):
    """c1 = (k-1)/(k+1) multiplying the A_R term and c2 = 2k/(k+1) multiplying R (Def. 4.1)."""
    return (k - 1.0) / (k + 1.0), 2.0 * k / (k + 1.0)


def n_hss(k, theta=1.0):
    """Number of inner HSS iterations ceil(k^theta) (Def. 4.1 with m ceil(k); Sec. 5.2)."""
    val = float(k) ** float(theta)
    r = round(val)
    if abs(val - r) <= 1e-9 * max(1.0, val):
        return int(r)
    return int(math.ceil(val))


def combine(mats, coeff):
    K, M, MG = mats
    cK, cM, cG = coeff
    return (cK * K + cM * M + cG * MG).tocsr()


# ---------------------------------------------------------------------------
# Grid transfer: P[f, c] = coarse hat function c evaluated at fine node f
# ---------------------------------------------------------------------------
def prolongation(fine):
    """Bi/trilinear interpolation from ``fine.coarse()`` to ``fine`` (coarse -> fine).

    Built entrywise from the definition of the nested Q1 spaces: column c holds
    the coarse basis function of node c sampled at the fine nodes.  Rows of fine
    Dirichlet nodes and columns of coarse Dirichlet nodes are zero.
    """
    coarse = fine.coarse()
    dim = fine.dim
    ijk = fine.node_ijk()
    rows, cols, vals = [], [], []
    # candidate coarse indices per axis: floor and ceil of i_f / 2
    choices = []
    for ax in range(dim):
        i = ijk[:, ax]
        choices.append((i // 2, (i + 1) // 2))
    for pick in np.ndindex(*([2] * dim)):
        ci = [choices[ax][pick[ax]] for ax in range(dim)]
        # skip duplicates when floor == ceil (even fine index): keep pick 0 only
        keep = np.ones(fine.N, dtype=bool)
        w = np.ones(fine.N)
        for ax in range(dim):
            if pick[ax] == 1:
                keep &= choices[ax][0] != choices[ax][1]
            xf = ijk[:, ax] * fine.h
            xc = ci[ax] * coarse.h
            w = w * np.maximum(0.0, 1.0 - np.abs(xf - xc) / coarse.h)
        sel = keep & (w != 0.0)
        rows.append(np.nonzero(sel)[0])
        cols.append(coarse.index(*[c[sel] for c in ci]))
        vals.append(w[sel])
    P = sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                      shape=(fine.N, coarse.N))
    P = (sp.diags(fine.free().astype(float)) @ P @ sp.diags(coarse.free().astype(float))).tocsr()
    P.eliminate_zeros()
    return P


# ---------------------------------------------------------------------------
# Problem: hierarchy of operators
# ---------------------------------------------------------------------------
@dataclass
class Options:
    """Multigrid / outer-solver settings (names follow the paper where it has them)."""

    theta: float = 1.0          # ceil(k^theta) inner HSS iterations (Sec. 5.2)
    levels: int = 4             # 4 levels, coarsening factor 2 (Sec. 5.3)
    nu_pre: int = 2
    nu_post: int = 2
    nu_coarse: int = 8
    omega: float = 0.0          # Jacobi damping; 0 = 0.6 in 2D, 0.5 in 3D
    cycles_per_hss: int = 1
    gamma: int = 1              # cycle index: 1 V-cycle, 2 W-cycle (Sec. 5.3 uses a W-cycle)
    smoother: str = "jacobi"    # "jacobi": nu scaled-Jacobi sweeps; "gmres": nu iterations of
                                # GMRES with a Jacobi preconditioner (Sec. 5.3's smoother)
    restart: int = 30
    max_outer: int = 200


@dataclass
class Problem:
    grid: Grid
    k: float
    delta: float
    delta_hat: float
    opts: Options = field(default_factory=Options)
    al_coeff: tuple = None      # (c_K, c_M, c_G) of the operator the inner cycles solve; default
                                # A_L of Def. 4.1 (the mixed formulation passes its own, Def. 4.2)

    def __post_init__(self):
        if self.k <= 0 or self.delta < 0 or self.delta_hat <= 0:
            raise ValueError("need k > 0, delta >= 0, delta_hat > 0")
        L = self.opts.levels
        if self.grid.n % (2 ** (L - 1)):
            raise ValueError("n must be divisible by 2^(levels-1)")
        if self.opts.omega == 0.0:
            # damping by dimension: D^{-1}M reaches 9/4 in 2D and 27/8 in 3D, and the
            # shifted mass term dominates A_L on coarse levels, so 3D needs omega < 0.59
            self.opts = Options(**{**self.opts.__dict__, "omega": 0.5 if self.grid.dim == 3 else 0.6})
        self.grids = [self.grid]
        for _ in range(L - 1):
            self.grids.append(self.grids[-1].coarse())
        self.mats = [assemble(g) for g in self.grids]
        self.P = [prolongation(self.grids[l]) for l in range(L - 1)]
        cal = self.al_coeff if self.al_coeff is not None else coeff_AL(self.k, self.delta_hat)
        self.AL = [combine(m, cal) for m in self.mats]
        self.AR0 = combine(self.mats[0], coeff_AR(self.k, self.delta_hat))
        self.B = combine(self.mats[0], coeff_B(self.k, self.delta))
        self.free = [g.free() for g in self.grids]
        self.Dinv = []
        for l, A in enumerate(self.AL):
            d = A.diagonal().copy()
            d[~self.free[l]] = 1.0
            dinv = 1.0 / d
            dinv[~self.free[l]] = 0.0
            self.Dinv.append(dinv)
        self.counters = {"vcycles": 0, "hss": 0}

    # -- multigrid ----------------------------------------------------------
    def jacobi(self, l, b, x):
        """One scaled-Jacobi sweep x <- x + omega D^{-1} (b - A_L x), D = diag(A_L)."""
        return x + self.opts.omega * self.Dinv[l] * (b - self.AL[l] @ x)

    def gmres_smooth(self, l, b, x, s):
        """s iterations of GMRES on the Jacobi-preconditioned system D^{-1} A_L x = D^{-1} b
        of level l, started from x, without restart (the smoother of Sec. 5.3; preconditioner
        applied on the left, D = diag(A_L)).  The result is x + V y, where the columns of V
        are an orthonormal basis of the Krylov space K_s(D^{-1} A_L, z0), z0 = D^{-1}(b - A_L x),
        and y minimises ||D^{-1}(b - A_L (x + V y))||_2 = ||beta e1 - H y||_2 (Arnoldi relation
        D^{-1} A_L V_s = V_{s+1} H).  Arnoldi by modified Gram-Schmidt; the small least-squares
        problem by numpy's lstsq.  The loop stops early at a breakdown (h_{j+1,j} = 0 up to
        rounding: the Krylov space is invariant and the minimiser solves the system)."""
        A, dinv = self.AL[l], self.Dinv[l]
        z0 = dinv * (b - A @ x)
        beta = np.linalg.norm(z0)
        if s == 0 or beta == 0.0:
            return x
        V = [z0 / beta]
        H = np.zeros((s + 1, s), dtype=complex)
        m = s
        for j in range(s):
            w = dinv * (A @ V[j])
            for i in range(j + 1):
                H[i, j] = np.vdot(V[i], w)
                w = w - H[i, j] * V[i]
            H[j + 1, j] = np.linalg.norm(w)
            if H[j + 1, j].real <= 1e-14 * beta:
                m = j + 1
                break
            V.append(w / H[j + 1, j])
        rhs = np.zeros(m + 1, dtype=complex)
        rhs[0] = beta
        y = np.linalg.lstsq(H[:m + 1, :m], rhs, rcond=None)[0]
        return x + sum(y[i] * V[i] for i in range(m))

    def smooth(self, l, b, x, nu):
        """nu smoothing steps on level l: scaled-Jacobi sweeps, or GMRES(nu) with Jacobi."""
        if self.opts.smoother == "gmres":
            return self.gmres_smooth(l, b, x, nu)
        for _ in range(nu):
            x = self.jacobi(l, b, x)
        return x

    def vcycle(self, l, b):
        """One multigrid cycle on A_L of level l from the zero initial guess (returns x):
        a V-cycle for gamma = 1; for gamma = 2 (W-cycle) the coarse correction is two cycles
        on the coarse problem, the second on the residual the first leaves."""
        o = self.opts
        x = np.zeros_like(b)
        if l == len(self.AL) - 1:
            return self.smooth(l, b, x, o.nu_coarse)
        x = self.smooth(l, b, x, o.nu_pre)
        rc = self.P[l].T @ (b - self.AL[l] @ x)
        ec = self.vcycle(l + 1, rc)
        for _ in range(o.gamma - 1):
            ec = ec + self.vcycle(l + 1, rc - self.AL[l + 1] @ ec)
        x = x + self.P[l] @ ec
        return self.smooth(l, b, x, o.nu_post)

    def mg_solve(self, b):
        """cycles_per_hss V-cycles for A_L x = b starting from x = 0."""
        x = self.vcycle(0, b)
        self.counters["vcycles"] += 1
        for _ in range(self.opts.cycles_per_hss - 1):
            x = x + self.vcycle(0, b - self.AL[0] @ x)
            self.counters["vcycles"] += 1
        return x

    # -- HSS ------------------------------------------------------------------
    def hss_rhs(self, u, r):
        """c1 A_R u + c2 r, the right side of Def. 4.1."""
        c1, c2 = hss_weights(self.k)
        return c1 * (self.AR0 @ u) + c2 * r

    def prec(self, r, inner=None):
        """Shifted-HSS preconditioner of Def. 4.1: u_0 = 0, ceil(k^theta) HSS steps.

        ``inner`` solves A_L x = rhs; default is the multigrid approximation.
        """
        solve = self.mg_solve if inner is None else inner
        u = np.zeros_like(r)
        for _ in range(n_hss(self.k, self.opts.theta)):
            u = solve(self.hss_rhs(u, r))
            self.counters["hss"] += 1
        return u

    # -- exact --------------------------------------------------------------
    def lu(self, which="B"):
        """Sparse LU of the free-DoF block of B_delta (``"B"``) or A_L (``"AL"``)."""
        A = self.B if which == "B" else self.AL[0]
        f = np.nonzero(self.free[0])[0]
        lu = spla.splu(A[f][:, f].tocsc())

        def solve(b):
            x = np.zeros(self.grid.N, dtype=complex)
            x[f] = lu.solve(np.asarray(b, dtype=complex)[f])
            return x

        return solve


def fgmres(apply_A, b, prec, tol, restart=30, max_it=200, x0=None):
    """Right-preconditioned flexible GMRES (Saad 1993) with modified Gram-Schmidt.

    Stops when the Givens residual estimate drops below tol * ||b|| and the true
    residual ||b - A x|| / ||b||, recomputed at the end of each cycle, is <= tol.
    Returns (x, iterations, true relative residual, history of estimates).
    """
    b = np.asarray(b, dtype=complex)
    x = np.zeros_like(b) if x0 is None else np.array(x0, dtype=complex)
    bnorm = np.linalg.norm(b)
    if bnorm == 0.0:
        return np.zeros_like(b), 0, 0.0, []
    its = 0
    hist = []
    r = b - apply_A(x)
    while True:
        beta = np.linalg.norm(r)
        if beta / bnorm <= tol or its >= max_it:
            return x, its, beta / bnorm, hist
        m = restart
        V = np.zeros((m + 1, b.size), dtype=complex)
        Z = np.zeros((m, b.size), dtype=complex)
        H = np.zeros((m + 1, m), dtype=complex)
        cs = np.zeros(m)
        sn = np.zeros(m, dtype=complex)
        g = np.zeros(m + 1, dtype=complex)
        g[0] = beta
        V[0] = r / beta
        j_end = 0
        for j in range(m):
            Z[j] = prec(V[j])
            w = apply_A(Z[j])
            for i in range(j + 1):
                H[i, j] = np.vdot(V[i], w)
                w = w - H[i, j] * V[i]
            H[j + 1, j] = np.linalg.norm(w)
            if H[j + 1, j] != 0.0:
                V[j + 1] = w / H[j + 1, j]
            for i in range(j):  # previous rotations
                t = cs[i] * H[i, j] + sn[i] * H[i + 1, j]
                H[i + 1, j] = -np.conj(sn[i]) * H[i, j] + cs[i] * H[i + 1, j]
                H[i, j] = t
            h1, h2 = H[j, j], H[j + 1, j]
            den = math.hypot(abs(h1), abs(h2))
            if abs(h1) == 0.0:
                cs[j], sn[j] = 0.0, 1.0
            else:
                cs[j] = abs(h1) / den
                sn[j] = (h1 / abs(h1)) * np.conj(h2) / den
            H[j, j] = cs[j] * h1 + sn[j] * h2
            H[j + 1, j] = 0.0
            g[j + 1] = -np.conj(sn[j]) * g[j]
            g[j] = cs[j] * g[j]
            its += 1
            j_end = j + 1
            hist.append(abs(g[j + 1]) / bnorm)
            if abs(g[j + 1]) / bnorm <= tol or its >= max_it:
                break
        # back substitution for y, then x += Z^T y
        y = np.zeros(j_end, dtype=complex)
        for i in range(j_end - 1, -1, -1):
            y[i] = (g[i] - H[i, i + 1:j_end] @ y[i + 1:]) / H[i, i]
        x = x + y @ Z[:j_end]
        r = b - apply_A(x)


def solve(prob: Problem, b, tol, x0=None, inner=None):
    """Outer FGMRES on B_delta u = b preconditioned by the shifted-HSS operator (Sec. 5.1)."""
    A = prob.B
    return fgmres(lambda v: A @ v, b, lambda v: prob.prec(v, inner=inner), tol,
                  restart=prob.opts.restart, max_it=prob.opts.max_outer, x0=x0)


def richardson(apply_A, b, prec, tol, max_it=200, x0=None):
    """Preconditioned Richardson (stationary) iteration u^{n+1} = u^n + P(b - A u^n), the
    iteration that the text after Def. 4.1 defines with P the shifted-HSS preconditioner.

    Stops when the true relative residual ||b - A u|| / ||b|| (computed every step) is
    <= tol.  Returns (x, iterations, relative residual, history of residuals).
    """
    b = np.asarray(b, dtype=complex)
    x = np.zeros_like(b) if x0 is None else np.array(x0, dtype=complex)
    bnorm = np.linalg.norm(b)
    if bnorm == 0.0:
        return np.zeros_like(b), 0, 0.0, []
    r = b - apply_A(x)
    rel = np.linalg.norm(r) / bnorm
    hist = [rel]
    its = 0
    while rel > tol and its < max_it:
        x = x + prec(r)
        r = b - apply_A(x)
        rel = np.linalg.norm(r) / bnorm
        hist.append(rel)
        its += 1
    return x, its, rel, hist


def solve_richardson(prob: Problem, b, tol, x0=None, inner=None):
    """Outer preconditioned Richardson on B_delta u = b with the shifted-HSS operator."""
    A = prob.B
    return richardson(lambda v: A @ v, b, lambda v: prob.prec(v, inner=inner), tol,
                      max_it=prob.opts.max_outer, x0=x0)


def load_vector_nodal(grid, f_nodal):
    """b = M f for a nodal interpolant f (the right side G[v] of Sec. 2 with f in Q1)."""
    _, M, _ = assemble(grid)
    return M @ np.asarray(f_nodal, dtype=complex)


def load_vector_quadrature(grid, f, nq=3):
    """b_v = int f phi_v by tensor Gauss-Legendre quadrature (nq points per axis per cell)."""
    dim, h = grid.dim, grid.h
    xg, wg = np.polynomial.legendre.leggauss(nq)
    xg = 0.5 * (xg + 1.0)
    wg = 0.5 * wg
    cells, g = _cell_vertex_globals(grid)
    b = np.zeros(grid.N, dtype=complex)
    nodes = _local_nodes(dim)
    for q in np.ndindex(*([nq] * dim)):
        xi = [xg[qi] for qi in q]
        w = np.prod([wg[qi] for qi in q]) * h ** dim
        pts = [(cells[:, d] + xi[d]) * h for d in range(dim)]
        fv = f(*pts)
        for A, a in enumerate(nodes):
            np.add.at(b, g[:, A], w * fv * _phi(a, xi))
    b[~grid.free()] = 0.0
    return b


def q1_errors(grid, u_nodal, u_exact, grad_exact, nq=3):
    """L2 and H1-seminorm errors of the Q1 function with nodal values u_nodal."""
    dim, h = grid.dim, grid.h
    xg, wg = np.polynomial.legendre.leggauss(nq)
    xg = 0.5 * (xg + 1.0)
    wg = 0.5 * wg
    cells, g = _cell_vertex_globals(grid)
    nodes = _local_nodes(dim)
    e0 = 0.0
    e1 = 0.0
    for q in np.ndindex(*([nq] * dim)):
        xi = [xg[qi] for qi in q]
        w = np.prod([wg[qi] for qi in q]) * h ** dim
        pts = [(cells[:, d] + xi[d]) * h for d in range(dim)]
        uh = np.zeros(cells.shape[0], dtype=complex)
        guh = [np.zeros(cells.shape[0], dtype=complex) for _ in range(dim)]
        for A, a in enumerate(nodes):
            ua = u_nodal[g[:, A]]
            uh += ua * _phi(a, xi)
            for ax in range(dim):
                guh[ax] += ua * _dphi(a, xi, ax) / h
        e0 += w * np.sum(np.abs(uh - u_exact(*pts)) ** 2)
        ge = grad_exact(*pts)
        e1 += w * sum(np.sum(np.abs(guh[ax] - ge[ax]) ** 2) for ax in range(dim))
    return math.sqrt(e0), math.sqrt(e1)
