"""Pins of the FP64 oracle against facts that the paper and the mathematics fix.

Each test checks the oracle against something other than itself: closed forms,
exact integrals of functions that lie in the Q1 space, an independent Kronecker
construction, identities proved in the paper (Prop. 3.2, Cor. 3.3), a dense
matrix formula, values printed in the paper (tests/golden), manufactured
solutions, and sparse LU.
"""
import math
import os

import numpy as np
import pytest
import scipy.linalg as sla
import scipy.sparse as sp

from oracle import hh_oracle as O
from paper_2506_18694_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
S, D = O.SOMMERFELD, O.DIRICHLET


def _ones(g):
    return np.ones(g.N)


def _interp(g, fun):
    x = g.coords()
    return fun(*[x[:, d] for d in range(g.dim)])


# --------------------------------------------------------------------- P1
@pytest.mark.parametrize("dim,n", [(2, 4), (2, 7), (3, 3)])
def test_p1_symmetry_and_definiteness(dim, n):
    g = O.Grid(dim, n, (S,) * (2 * dim))
    K, M, MG = O.assemble(g)
    for A in (K, M, MG):
        assert abs(A - A.T).max() < 1e-15
    Md = M.toarray()
    np.linalg.cholesky(Md)  # M is SPD
    ev = np.linalg.eigvalsh(K.toarray())
    assert ev.min() > -1e-12  # K is PSD
    assert np.abs(K @ _ones(g)).max() < 1e-13  # constants are in the kernel of K


@pytest.mark.parametrize("dim,n", [(2, 4), (2, 6), (3, 2), (3, 4)])
def test_p1_exact_integrals(dim, n):
    """Integrals of functions that Q1 reproduces exactly on the unit square / cube."""
    g = O.Grid(dim, n, (S,) * (2 * dim))
    K, M, MG = O.assemble(g)
    one = _ones(g)
    assert abs(one @ M @ one - 1.0) < 1e-13               # |Omega|
    assert abs(one @ MG @ one - 2 * dim) < 1e-13          # |boundary| = 4 or 6
    for ax in range(dim):
        x = g.coords()[:, ax]
        assert abs(x @ K @ x - 1.0) < 1e-13                # int |grad x|^2
    prod = np.prod(g.coords(), axis=1)                     # x y (z): in Q1
    if dim == 2:
        assert abs(prod @ K @ prod - 2.0 / 3.0) < 1e-13    # int x^2 + y^2
        assert abs(prod @ M @ prod - 1.0 / 9.0) < 1e-13    # int x^2 y^2
        assert abs(prod @ MG @ prod - 2.0 / 3.0) < 1e-13   # sides x=1, y=1: int t^2
    else:
        assert abs(prod @ K @ prod - 1.0 / 3.0) < 1e-13
        assert abs(prod @ M @ prod - 1.0 / 27.0) < 1e-13
        assert abs(prod @ MG @ prod - 1.0 / 3.0) < 1e-13   # three faces at 1: int s^2 t^2


def test_p1_dirichlet_masking():
    g = O.Grid(3, 4, (S, S, S, S, D, S))
    K, M, MG = O.assemble(g)
    dn = g.dirichlet_nodes()
    assert dn.sum() == 25
    for A in (K, M, MG):
        assert abs(A[dn]).max() == 0 and abs(A[:, dn]).max() == 0
    # full all-Sommerfeld matrices restricted to free nodes coincide
    g2 = O.Grid(3, 4, (S, S, S, S, S, S))
    K2, M2, _ = O.assemble(g2)
    f = ~dn
    assert abs(K[f][:, f] - K2[f][:, f]).max() < 1e-15
    assert abs(M[f][:, f] - M2[f][:, f]).max() < 1e-15


# --------------------------------------------------------------------- P2
def _global_1d(n):
    h = 1.0 / n
    K1 = sp.diags([-np.ones(n), 2 * np.ones(n + 1), -np.ones(n)], [-1, 0, 1]).tolil() / h
    M1 = sp.diags([np.ones(n), 4 * np.ones(n + 1), np.ones(n)], [-1, 0, 1]).tolil() * (h / 6)
    K1[0, 0] = K1[n, n] = 1.0 / h
    M1[0, 0] = M1[n, n] = h / 3.0
    return K1.tocsr(), M1.tocsr()


@pytest.mark.parametrize("dim,n", [(2, 5), (3, 4)])
def test_p2_kronecker_form(dim, n):
    g = O.Grid(dim, n, (S,) * (2 * dim))
    K, M, MG = O.assemble(g)
    K1, M1 = _global_1d(n)
    I1 = sp.identity(n + 1)
    e0 = sp.csr_matrix(([1.0], ([0], [0])), shape=(n + 1, n + 1))
    en = sp.csr_matrix(([1.0], ([n], [n])), shape=(n + 1, n + 1))
    if dim == 2:  # node index i + (n+1) j  ->  kron(y-factor, x-factor)
        Kk = sp.kron(M1, K1) + sp.kron(K1, M1)
        Mk = sp.kron(M1, M1)
        MGk = sp.kron(M1, e0 + en) + sp.kron(e0 + en, M1)
    else:
        Kk = (sp.kron(sp.kron(M1, M1), K1) + sp.kron(sp.kron(M1, K1), M1)
              + sp.kron(sp.kron(K1, M1), M1))
        Mk = sp.kron(sp.kron(M1, M1), M1)
        MGk = (sp.kron(sp.kron(M1, M1), e0 + en) + sp.kron(sp.kron(M1, e0 + en), M1)
               + sp.kron(sp.kron(e0 + en, M1), M1))
    assert abs(K - Kk).max() < 1e-12
    assert abs(M - Mk).max() < 1e-15
    assert abs(MG - MGk).max() < 1e-15
    del I1


# --------------------------------------------------------------------- P3
@pytest.mark.parametrize("dim,n,bc", [(2, 8, (S, S, S, S)), (2, 8, (D, S, S, D)),
                                      (3, 4, (S, S, S, S, D, S)), (3, 4, (D, D, S, S, S, D))])
def test_p3_galerkin_identity(dim, n, bc):
    gf = O.Grid(dim, n, bc)
    P = O.prolongation(gf)
    for Af, Ac in zip(O.assemble(gf), O.assemble(gf.coarse())):
        assert abs(P.T @ Af @ P - Ac).max() < 1e-13


@pytest.mark.parametrize("dim", [2, 3])
def test_p3_prolongation_reproduces_multilinear(dim):
    gf = O.Grid(dim, 8, (S,) * (2 * dim))
    gc = gf.coarse()
    fun = (lambda x, y: 1 + 2 * x - 3 * y + 5 * x * y) if dim == 2 else \
          (lambda x, y, z: 1 + x - y + 2 * z + x * y * z - 4 * y * z)
    P = O.prolongation(gf)
    assert abs(P @ _interp(gc, fun) - _interp(gf, fun)).max() < 1e-13
    # every row of P sums to one (partition of unity) when there is no Dirichlet side
    assert abs(P @ np.ones(gc.N) - 1).max() < 1e-15


# --------------------------------------------------------------------- P4
@pytest.mark.parametrize("k,dh", [(6.0, 2.0), (10.0, 10.0), (7.5, 0.5)])
def test_p4_cayley_h_unitary(k, dh):
    """y = A_L^{-1} A_R x preserves the H norm, H = 2 dh k M + k M_Gamma (proof of Prop. 3.2)."""
    g = O.Grid(2, 8, (S, S, D, S))
    mats = O.assemble(g)
    AL = O.combine(mats, O.coeff_AL(k, dh)).toarray()
    AR = O.combine(mats, O.coeff_AR(k, dh)).toarray()
    H = O.combine(mats, O.coeff_H(k, dh)).toarray().real
    f = g.free()
    AL, AR, H = AL[f][:, f], AR[f][:, f], H[f][:, f]
    rng = np.random.default_rng(1)
    for _ in range(3):
        x = rng.standard_normal(f.sum()) + 1j * rng.standard_normal(f.sum())
        y = np.linalg.solve(AL, AR @ x)
        nx = np.real(np.conj(x) @ H @ x)
        ny = np.real(np.conj(y) @ H @ y)
        assert abs(ny - nx) <= 1e-12 * nx


@pytest.mark.parametrize("k,dh", [(10.0, 2.0), (80.0, 80.0), (3.3, 0.7)])
def test_p4_fixed_point_is_shifted_operator(k, dh):
    """A_L - c1 A_R = c2 B_dh: the HSS fixed point solves B_dh u = R (Def. 4.1)."""
    g = O.Grid(2, 4, (S, D, S, S))
    mats = O.assemble(g)
    c1, c2 = O.hss_weights(k)
    lhs = O.combine(mats, O.coeff_AL(k, dh)) - c1 * O.combine(mats, O.coeff_AR(k, dh))
    rhs = c2 * O.combine(mats, O.coeff_B(k, dh))
    assert abs(lhs - rhs).max() <= 1e-12 * abs(rhs).max()


def test_p4_shifted_operator_matches_form():
    """B_delta = K + (-delta + i k)^2 M - (-delta + i k) M_Gamma, by the weak form of Sec. 2."""
    k, delta = 7.0, 0.3
    cK, cM, cG = O.coeff_B(k, delta)
    assert cK == 1.0
    assert abs(cM - (delta ** 2 - k ** 2 - 2j * delta * k)) < 1e-12
    assert abs(cG - (delta - 1j * k)) < 1e-15


# --------------------------------------------------------------------- P5 / P9 (golden)
def _golden(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as fh:
        for line in fh:
            if line.strip() and not line.startswith("#"):
                rows.append([float(t) for t in line.split()])
    return np.array(rows)


def test_golden_table5_nu_s():
    """nu_s printed in Table 5 equals the HSS contraction factor (k-1)/(k+1) of Prop. 3.2."""
    for k, nu_s, _ in _golden("table5_hss_rate.txt"):
        c1, _ = O.hss_weights(k)
        assert abs(c1 - nu_s) <= 0.5e-4


def test_golden_table1_hss_counts():
    """Bracketed totals of Table 1 divided by the outer count are ceil(k^theta)."""
    for k, theta, outer, total in _golden("table1_hss_counts.txt"):
        assert O.n_hss(k, theta) * outer == total
    assert O.n_hss(80.0) == 80 and O.n_hss(40.0) == 40 and O.n_hss(10.5) == 11


def _hss_errors(prob, R, steps):
    """H-norm errors of the exact-inner-solve HSS iteration against B_dh^{-1} R."""
    k, dh = prob.k, prob.delta_hat
    lu_AL = prob.lu("AL")
    Bdh = O.combine(prob.mats[0], O.coeff_B(k, dh))
    f = np.nonzero(prob.free[0])[0]
    import scipy.sparse.linalg as spla
    ustar = np.zeros(prob.grid.N, dtype=complex)
    ustar[f] = spla.spsolve(Bdh[f][:, f].tocsc(), R[f])
    H = O.combine(prob.mats[0], O.coeff_H(k, dh))
    u = np.zeros_like(R)
    errs = []
    for _ in range(steps):
        e = u - ustar
        errs.append(math.sqrt(np.real(np.conj(e) @ (H @ e))))
        u = lu_AL(prob.hss_rhs(u, R))
    e = u - ustar
    errs.append(math.sqrt(np.real(np.conj(e) @ (H @ e))))
    return np.array(errs)


@pytest.mark.parametrize("k,n,dh", [(8.0, 16, 2.0), (16.0, 32, 2.0), (10.0, 16, 10.0)])
def test_p5_hss_contraction_every_step(k, n, dh):
    """Prop. 3.2: ||e_{n+1}||_H <= (k-1)/(k+1) ||e_n||_H at every step (exact inner solves)."""
    g = O.Grid(2, n, (S,) * 4)
    prob = O.Problem(g, k, 0.0, dh, O.Options(levels=1))
    rng = np.random.default_rng(3)
    R = (rng.standard_normal(g.N) + 1j * rng.standard_normal(g.N)) * g.free()
    errs = _hss_errors(prob, R, O.n_hss(k))
    nu = O.hss_weights(k)[0]
    ratios = errs[1:] / errs[:-1]
    assert np.all(ratios <= nu * (1 + 1e-10))
    # Cor. 3.3 with m = 1: ceil(k) steps reduce the H-norm error by at least e^{-1}
    assert errs[-1] <= math.exp(-1.0) * errs[0]
    # the bound is close to tight (Table 5 reports eta_s within 1% of nu_s)
    assert ratios[-1] > 0.9 * nu


def test_p5_hss_iteration_count_grows_linearly_in_k():
    """The O(k) growth that Prop. 3.2 implies: the exact-inner-solve HSS steps needed for a
    fixed H-norm error reduction (1e-3) stay under the bound ln(1e3) / ln(1 / nu_s), and double
    with k (10 points per wavelength or more, delta_hat = 2)."""
    counts = {}
    for k, n in ((8.0, 16), (16.0, 32), (32.0, 64)):
        g = O.Grid(2, n, (S,) * 4)
        prob = O.Problem(g, k, 0.0, 2.0, O.Options(levels=1))
        rng = np.random.default_rng(7)
        R = (rng.standard_normal(g.N) + 1j * rng.standard_normal(g.N)) * g.free()
        nu = O.hss_weights(k)[0]
        bound = math.ceil(math.log(1e3) / math.log(1.0 / nu))
        errs = _hss_errors(prob, R, bound)
        hit = np.nonzero(errs <= 1e-3 * errs[0])[0]
        assert hit.size, (k, errs[-1] / errs[0])
        counts[k] = int(hit[0])
        assert counts[k] <= bound
    for lo, hi in ((8.0, 16.0), (16.0, 32.0)):
        assert 1.6 <= counts[hi] / counts[lo] <= 2.4, counts


# --------------------------------------------------------------------- multigrid
def _dense_vcycle_operator(prob, l):
    """Approximate inverse B_l of one V-cycle from x = 0, as a dense matrix.

    Coarsest: sum_{i < nu_c} S^i omega D^{-1}.  Otherwise
    I - B_l A = S^{nu2} (I - P B_{l+1} P^T A) S^{nu1} with S = I - omega D^{-1} A.
    """
    o = prob.opts
    A = prob.AL[l].toarray()
    Dw = np.diag(o.omega * prob.Dinv[l])
    Sm = np.eye(A.shape[0]) - Dw @ A
    if l == len(prob.AL) - 1:
        B = np.zeros_like(A)
        Si = np.eye(A.shape[0])
        for _ in range(o.nu_coarse):
            B = B + Si @ Dw
            Si = Sm @ Si
        return B
    Bc = _dense_vcycle_operator(prob, l + 1)
    if o.gamma > 1:
        # gamma cycles on the coarse problem: sum_{m < gamma} (I - Bc Ac)^m Bc
        Ac = prob.AL[l + 1].toarray()
        G = np.eye(Ac.shape[0]) - Bc @ Ac
        Bc = sum(np.linalg.matrix_power(G, m) @ Bc for m in range(o.gamma))
    P = prob.P[l].toarray()
    E = np.linalg.matrix_power(Sm, o.nu_post) @ (np.eye(A.shape[0]) - P @ Bc @ P.T @ A) \
        @ np.linalg.matrix_power(Sm, o.nu_pre)
    free = np.diag(prob.free[l].astype(float))
    # restrict to the free space: B = (I - E) A^{-1} on free nodes
    f = prob.free[l]
    B = np.zeros_like(A)
    B[np.ix_(f, f)] = (free @ (np.eye(A.shape[0]) - E))[np.ix_(f, f)] @ np.linalg.inv(A[np.ix_(f, f)])
    return B


@pytest.mark.parametrize("gamma", [1, 2])
@pytest.mark.parametrize("bc", [(S, S, S, S), (D, S, S, D)])
def test_vcycle_matches_error_propagation_formula(bc, gamma):
    g = O.Grid(2, 8, bc)
    prob = O.Problem(g, 5.0, 0.0, 2.0, O.Options(levels=3, nu_pre=1, nu_post=2, nu_coarse=3, gamma=gamma))
    B = _dense_vcycle_operator(prob, 0)
    rng = np.random.default_rng(5)
    b = (rng.standard_normal(g.N) + 1j * rng.standard_normal(g.N)) * g.free()
    assert np.abs(prob.vcycle(0, b) - B @ b).max() <= 1e-11 * np.abs(B @ b).max()


@pytest.mark.parametrize("cycles", [1, 2, 3])
@pytest.mark.parametrize("bc", [(S, S, S, S), (D, S, S, D)])
def test_mg_solve_cycles_match_error_propagation_power(bc, cycles):
    """cycles_per_hss = c cycles per inexact A_L solve of the HSS step (Def. 4.1), each on the
    residual the previous ones leave, are the stationary iteration x <- x + B (b - A x) from 0:
    the error after c cycles is (I - B A)^c e_0, so x = (I - (I - B A)^c) A^{-1} b on the free
    nodes, with B the dense single-cycle operator above."""
    g = O.Grid(2, 8, bc)
    prob = O.Problem(g, 5.0, 0.0, 2.0,
                     O.Options(levels=3, nu_pre=1, nu_post=2, nu_coarse=3, cycles_per_hss=cycles))
    B = _dense_vcycle_operator(prob, 0)
    A = prob.AL[0].toarray()
    f = prob.free[0]
    rng = np.random.default_rng(11 + cycles)
    b = (rng.standard_normal(g.N) + 1j * rng.standard_normal(g.N)) * g.free()
    x_exact = np.zeros(g.N, dtype=complex)
    x_exact[f] = np.linalg.solve(A[np.ix_(f, f)], b[f])
    E = np.eye(g.N) - B @ A
    want = x_exact - np.linalg.matrix_power(E, cycles) @ x_exact
    got = prob.mg_solve(b)
    assert np.abs(got - want).max() <= 1e-10 * np.abs(want).max()
    assert np.all(got[~f] == 0)
    assert prob.counters["vcycles"] == cycles


def test_vcycle_contracts_shifted_operator():
    """The V-cycle is a convergent approximate inverse of A_L at the default settings."""
    g = O.Grid(2, 64, (S,) * 4)
    prob = O.Problem(g, 10.0, 0.0, 2.0)
    rng = np.random.default_rng(6)
    e = (rng.standard_normal(g.N) + 1j * rng.standard_normal(g.N))
    b = prob.AL[0] @ e
    x = prob.mg_solve(b)
    assert np.linalg.norm(b - prob.AL[0] @ x) < 0.1 * np.linalg.norm(b)


# --------------------------------------------------------------------- FGMRES
def test_fgmres_dense_system():
    rng = np.random.default_rng(7)
    n = 40
    A = np.eye(n) * 4 + rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
    b = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    x, its, res, hist = O.fgmres(lambda v: A @ v, b, lambda v: v, 1e-12, restart=50, max_it=50)
    assert res <= 1e-12
    assert np.abs(x - np.linalg.solve(A, b)).max() < 1e-10
    assert np.all(np.diff(hist) <= 1e-14)  # GMRES residual never increases
    # restarted runs reach the same answer on a matrix whose field of values avoids 0
    A2 = 10 * np.eye(n) + 0.5 * (rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n)))
    x1, _, _, _ = O.fgmres(lambda v: A2 @ v, b, lambda v: v, 1e-13, restart=50, max_it=50)
    x2, its2, res2, _ = O.fgmres(lambda v: A2 @ v, b, lambda v: v, 1e-12, restart=3, max_it=400)
    assert res2 <= 1e-12 and np.abs(x2 - x1).max() < 1e-10 * np.abs(x1).max()
    assert np.abs(x1 - np.linalg.solve(A2, b)).max() < 1e-11 * np.abs(x1).max()


def test_fgmres_exact_preconditioner_one_step():
    rng = np.random.default_rng(8)
    n = 20
    A = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n)) + 5 * np.eye(n)
    Ainv = np.linalg.inv(A)
    b = rng.standard_normal(n) + 0j
    x, its, res, _ = O.fgmres(lambda v: A @ v, b, lambda v: Ainv @ v, 1e-12)
    assert its == 1 and res < 1e-12


# --------------------------------------------------------------------- P6
@pytest.mark.parametrize("dim,n,k,dh,bc", [
    (2, 32, 10.0, 10.0, (S,) * 4),
    (2, 32, 10.0, 2.0, (S,) * 4),
    (2, 16, 6.0, 2.0, (D, S, S, S)),
    (3, 8, 4.0, 2.0, (S, S, S, S, D, S)),
])
def test_p6_solver_matches_lu(dim, n, k, dh, bc):
    g = O.Grid(dim, n, bc)
    prob = O.Problem(g, k, 0.0, dh, O.Options(levels=3 if n >= 16 else 2))
    x = g.coords()
    f = np.exp(-((x - 0.5) ** 2).sum(1) / (2 * 0.05 ** 2)).astype(complex)
    b = O.load_vector_nodal(g, f)
    u, its, res, _ = O.solve(prob, b, 1e-10)
    ex = prob.lu("B")(b)
    assert res <= 1e-10
    assert np.linalg.norm(u - ex) <= 1e-7 * np.linalg.norm(ex)
    if (~g.free()).any():
        assert np.abs(u[~g.free()]).max() == 0.0


# --------------------------------------------------------------------- P7
def _manufactured_2d(k, delta):
    s = -delta + 1j * k

    def u(x, y):
        return (x * (1 - x) * y * (1 - y)) ** 2 + 0j

    def grad(x, y):
        px, py = (x * (1 - x)) ** 2, (y * (1 - y)) ** 2
        dpx = 2 * x * (1 - x) * (1 - 2 * x)
        dpy = 2 * y * (1 - y) * (1 - 2 * y)
        return [dpx * py + 0j, px * dpy + 0j]

    def f(x, y):
        px, py = (x * (1 - x)) ** 2, (y * (1 - y)) ** 2
        d2 = lambda t: 2 * (1 - 6 * t + 6 * t * t)  # second derivative of (t(1-t))^2
        lap = d2(x) * py + px * d2(y)
        return s * s * px * py - lap

    return u, grad, f


def test_p7_manufactured_convergence_rates():
    """Q1: L2 error ratio ~4 and H1 ratio ~2 per halving of h (zero boundary data)."""
    k, delta = 10.0, 0.5
    u, grad, f = _manufactured_2d(k, delta)
    errs = []
    for n in (16, 32, 64):
        g = O.Grid(2, n, (S, S, S, S))
        prob = O.Problem(g, k, delta, 1.0, O.Options(levels=1))
        b = O.load_vector_quadrature(g, f)
        uh = prob.lu("B")(b)
        errs.append(O.q1_errors(g, uh, u, grad))
    e = np.array(errs)
    r0 = e[:-1, 0] / e[1:, 0]
    r1 = e[:-1, 1] / e[1:, 1]
    assert np.all(r0 > 3.5) and np.all(r0 < 4.6)
    assert np.all(r1 > 1.8) and np.all(r1 < 2.2)


def test_p7_robin_boundary_term_convergence():
    """Inhomogeneous Sommerfeld data pins the boundary coefficient delta - i k of B_delta.

    u* = cos(pi x) cos(2 pi y) (smooth, nonzero on the boundary), delta = 0.4, k = 6.
    f = (-delta + i k)^2 u* + 5 pi^2 u*; g = du*/dn - (-delta + i k) u* on each side,
    and the load vector gains int_Gamma g phi_v dS.  Errors must fall at the Q1 rate.
    """
    k, delta = 6.0, 0.4
    s = -delta + 1j * k
    uex = lambda x, y: np.cos(np.pi * x) * np.cos(2 * np.pi * y) + 0j
    gex = lambda x, y: [-np.pi * np.sin(np.pi * x) * np.cos(2 * np.pi * y) + 0j,
                        -2 * np.pi * np.cos(np.pi * x) * np.sin(2 * np.pi * y) + 0j]
    fex = lambda x, y: (s * s + 5 * np.pi ** 2) * uex(x, y)
    errs = []
    for n in (16, 32, 64):
        g = O.Grid(2, n, (S, S, S, S))
        prob = O.Problem(g, k, delta, 1.0, O.Options(levels=1))
        b = O.load_vector_quadrature(g, fex)
        # boundary data: sides x=0 (n=-x), x=1 (n=+x), y=0 (n=-y), y=1 (n=+y)
        xg, wg = np.polynomial.legendre.leggauss(4)
        xg, wg = 0.5 * (xg + 1), 0.5 * wg
        h = g.h
        for side in range(4):
            ax, hi = side // 2, side % 2
            for c in range(n):
                for q, w in zip(xg, wg):
                    t = (c + q) * h
                    pt = [0.0, 0.0]
                    pt[ax] = 1.0 if hi else 0.0
                    pt[1 - ax] = t
                    gr = gex(*pt)
                    dudn = gr[ax] * (1 if hi else -1)
                    gval = dudn - s * uex(*pt)
                    ij = [0, 0]
                    ij[ax] = n if hi else 0
                    for a, phi in ((c, 1 - q), (c + 1, q)):
                        ij[1 - ax] = a
                        b[g.index(*ij)] += w * h * gval * phi
        uh = prob.lu("B")(b)
        errs.append(O.q1_errors(g, uh, uex, gex))
    e = np.array(errs)
    r0 = e[:-1, 0] / e[1:, 0]
    assert np.all(r0 > 3.5) and np.all(r0 < 4.6)
    assert e[-1, 0] < 1e-3


# --------------------------------------------------------------------- P8
@pytest.mark.parametrize("dim,n,bc", [(2, 32, (S,) * 4), (3, 8, (S, S, S, S, D, S))])
def test_p8_energy_identity(dim, n, bc):
    """delta = 0: Im(u^H b) = -k u^H M_Gamma u for the exact discrete solution."""
    g = O.Grid(dim, n, bc)
    k = 9.0
    prob = O.Problem(g, k, 0.0, 2.0, O.Options(levels=1))
    rng = np.random.default_rng(9)
    b = (rng.standard_normal(g.N) + 1j * rng.standard_normal(g.N)) * g.free()
    u = prob.lu("B")(b)
    MG = prob.mats[0][2]
    lhs = np.imag(np.vdot(u, b))
    rhs = -k * np.real(np.vdot(u, MG @ u))
    assert abs(lhs - rhs) <= 1e-10 * abs(rhs)


# --------------------------------------------------------------------- P9
def test_p9_theta_trend_outer_counts():
    """Outer FGMRES counts with exact inner solves follow the theta trend of Sec. 5.2.

    With ceil(k^theta) inner HSS steps, theta = 1/2 counts grow roughly like k^{1/2}
    while theta = 1 counts level off and theta = 3/2 needs no more than theta = 1
    (Tables 1-2 show the same trend for P1 triangles).
    """
    counts = {}
    for theta in (0.5, 1.0, 1.5):
        for k in (8.0, 16.0):
            n = int(8 * math.ceil(k ** 1.5 / 8))
            g = O.Grid(2, n, (S,) * 4)
            prob = O.Problem(g, k, 0.0, 2.0, O.Options(levels=1, theta=theta))
            inner = prob.lu("AL")
            b = O.load_vector_nodal(g, np.ones(g.N, dtype=complex))
            _, its, res, _ = O.solve(prob, b, 1e-6, inner=inner)
            assert res <= 1e-6
            counts[(theta, k)] = its
    for k in (8.0, 16.0):
        assert counts[(0.5, k)] > counts[(1.0, k)] >= counts[(1.5, k)]
    assert counts[(0.5, 16.0)] / counts[(0.5, 8.0)] > 1.6
    assert counts[(1.0, 16.0)] / counts[(1.0, 8.0)] < 1.35


def test_jacobi_sweeps_converge_to_lu():
    """Scaled Jacobi on a strongly shifted A_L (delta_hat = k) converges to the LU solution."""
    g = O.Grid(2, 16, (S, S, D, S))
    prob = O.Problem(g, 12.0, 0.0, 12.0, O.Options(levels=1, omega=0.6))
    rng = np.random.default_rng(10)
    b = (rng.standard_normal(g.N) + 1j * rng.standard_normal(g.N)) * g.free()
    x = np.zeros_like(b)
    for _ in range(300):
        x = prob.jacobi(0, b, x)
    ex = prob.lu("AL")(b)
    assert np.linalg.norm(x - ex) <= 1e-9 * np.linalg.norm(ex)


@pytest.mark.parametrize("dim,n,bc", [(2, 6, (S, D, S, S)), (3, 4, (S, S, S, S, D, S))])
def test_apply_elementwise_equals_assembled(dim, n, bc):
    """The matrix-free element loop applies the same operator as the assembled CSR matrix."""
    g = O.Grid(dim, n, bc)
    rng = np.random.default_rng(11)
    x = rng.standard_normal(g.N) + 1j * rng.standard_normal(g.N)
    for coeff in (O.coeff_AL(7.0, 2.0), O.coeff_B(7.0, 0.0), (1.0, 0.0, 0.0), (0.0, 0.0, 1.0)):
        ref = O.combine(O.assemble(g), coeff) @ (x * g.free())
        assert np.abs(O.apply_elementwise(g, coeff, x) - ref).max() <= 1e-12 * np.abs(ref).max()


@pytest.mark.parametrize("dim,n,bc", [(2, 5, (S, D, S, S)), (3, 3, (S, S, D, S, S, S))])
def test_diag_elementwise_equals_assembled(dim, n, bc):
    g = O.Grid(dim, n, bc)
    for coeff in (O.coeff_AL(7.0, 2.0), (1.0, 0.0, 0.0), (0.0, 1.0, 0.5)):
        ref = O.combine(O.assemble(g), coeff).diagonal()
        assert np.abs(O.diag_elementwise(g, coeff) - ref).max() <= 1e-13 * np.abs(ref).max()


def test_richardson_exact_preconditioner_one_step():
    """With P = A^{-1} the stationary iteration lands on the solution in one step."""
    rng = np.random.default_rng(41)
    A = rng.standard_normal((12, 12)) + 1j * rng.standard_normal((12, 12)) + 8 * np.eye(12)
    b = rng.standard_normal(12) + 1j * rng.standard_normal(12)
    Ainv = np.linalg.inv(A)
    x, its, rel, hist = O.richardson(lambda v: A @ v, b, lambda r: Ainv @ r, 1e-12)
    assert its == 1 and rel <= 1e-13
    assert np.allclose(x, np.linalg.solve(A, b), rtol=0, atol=1e-12)


def test_richardson_matches_neumann_series():
    """With a Jacobi preconditioner D^{-1}, step n equals sum_{m<n} (I - D^{-1}A)^m D^{-1} b."""
    rng = np.random.default_rng(42)
    n = 10
    A = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n)) + 12 * np.eye(n)
    b = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    Dinv = np.diag(1.0 / np.diag(A))
    x3, its, _, _ = O.richardson(lambda v: A @ v, b, lambda r: Dinv @ r, 0.0, max_it=3)
    G = np.eye(n) - Dinv @ A
    ref = sum(np.linalg.matrix_power(G, m) @ Dinv @ b for m in range(3))
    assert its == 3 and np.allclose(x3, ref, rtol=0, atol=1e-12)


def test_richardson_hss_converges_to_lu():
    """The HSS-preconditioned Richardson iteration (delta_hat = 2, each HSS step solved
    directly as in the paper's Richardson tables) converges monotonically to the LU solution
    (the contraction of Prop. 3.2 / Cor. 3.3 at work)."""
    g = O.Grid(2, 16, (O.SOMMERFELD,) * 4)
    f = inputs.gaussian_source(2, 16, (0.4, 0.6), 0.05)
    b = O.load_vector_nodal(g, f)
    prob = O.Problem(g, 6.0, 0.0, 2.0, O.Options(levels=2, max_outer=200))
    x, its, rel, hist = O.solve_richardson(prob, b, 1e-10, inner=prob.lu("AL"))
    ref = prob.lu("B")(b)
    assert rel <= 1e-10 and its < 200
    assert np.linalg.norm(x - ref) <= 1e-7 * np.linalg.norm(ref)
    assert all(h1 < h0 for h0, h1 in zip(hist, hist[1:]))


# --------------------------------------------------------------------- GMRES smoother
def _gmres_case(n, bc, seed):
    g = O.Grid(2, n, bc)
    prob = O.Problem(g, 6.0, 0.0, 3.0, O.Options(levels=1, smoother="gmres"))
    rng = np.random.default_rng(seed)
    b = (rng.standard_normal(g.N) + 1j * rng.standard_normal(g.N)) * g.free()
    x0 = (rng.standard_normal(g.N) + 1j * rng.standard_normal(g.N)) * g.free()
    return g, prob, b, x0


def test_gmres_smoother_full_krylov_space_solves():
    """With as many iterations as free unknowns the Krylov space is the whole free space, so
    GMRES from any starting vector returns the solution of A_L x = b (sparse LU)."""
    g, prob, b, x0 = _gmres_case(4, (S, D, S, S), 30)
    nf = int(g.free().sum())
    x = prob.gmres_smooth(0, b, x0, nf)
    ex = prob.lu("AL")(b)
    assert np.linalg.norm(x - ex) <= 1e-8 * np.linalg.norm(ex)


def test_gmres_smoother_one_step_closed_form():
    """One iteration is the minimal-residual step x0 + alpha z0 with z0 = D^{-1}(b - A x0),
    w = D^{-1} A z0 and alpha = (w^H z0) / (w^H w), the least-squares fit of z0 by w."""
    g, prob, b, x0 = _gmres_case(8, (S, S, D, S), 31)
    A, dinv = prob.AL[0], prob.Dinv[0]
    z0 = dinv * (b - A @ x0)
    w = dinv * (A @ z0)
    alpha = np.vdot(w, z0) / np.vdot(w, w)
    ref = x0 + alpha * z0
    assert np.linalg.norm(prob.gmres_smooth(0, b, x0, 1) - ref) <= 1e-12 * np.linalg.norm(ref)


def test_gmres_smoother_minimises_over_krylov_space():
    """After s = 3 iterations the preconditioned residual r is orthogonal to M K_3 (M = D^{-1} A,
    K_3 spanned by z0, M z0, M^2 z0: the normal equations of the minimisation), no larger than
    at other points of x0 + K_3 (random ones and three damped Jacobi sweeps), and it does not
    grow with the number of iterations."""
    g, prob, b, x0 = _gmres_case(8, (S, S, S, S), 32)
    A, dinv = prob.AL[0], prob.Dinv[0]
    M = lambda v: dinv * (A @ v)
    res = lambda x: dinv * (b - A @ x)
    z0 = res(x0)
    K = [z0, M(z0), M(M(z0))]
    x3 = prob.gmres_smooth(0, b, x0, 3)
    r3 = res(x3)
    for v in K:
        mv = M(v)
        assert abs(np.vdot(mv, r3)) <= 1e-10 * np.linalg.norm(mv) * np.linalg.norm(z0)
    rng = np.random.default_rng(33)
    for _ in range(30):
        c = rng.standard_normal(3) + 1j * rng.standard_normal(3)
        c *= 0.1 * np.linalg.norm(z0) / np.linalg.norm(c[0] * K[0] + c[1] * K[1] + c[2] * K[2])
        xc = x3 + c[0] * K[0] + c[1] * K[1] + c[2] * K[2]
        assert np.linalg.norm(r3) <= np.linalg.norm(res(xc)) * (1 + 1e-12)
    xj = x0
    for _ in range(3):
        xj = prob.jacobi(0, b, xj)
    assert np.linalg.norm(r3) <= np.linalg.norm(res(xj))
    norms = [np.linalg.norm(res(prob.gmres_smooth(0, b, x0, s))) for s in range(7)]
    assert all(norms[s + 1] <= norms[s] * (1 + 1e-12) for s in range(6))


def test_gmres_cycle_two_grid_exact_coarse_and_homogeneous():
    """A two-level cycle with no fine smoothing and GMRES on the coarse level with as many
    iterations as coarse unknowns is P A_c^{-1} P^T b exactly; the cycle with smoothing is
    homogeneous (b -> c b gives x -> c x for complex c), as GMRES is."""
    g = O.Grid(2, 8, (S, S, D, S))
    rng = np.random.default_rng(34)
    b = (rng.standard_normal(g.N) + 1j * rng.standard_normal(g.N)) * g.free()
    nfc = int(g.coarse().free().sum())
    prob = O.Problem(g, 6.0, 0.0, 3.0, O.Options(levels=2, nu_pre=0, nu_post=0, nu_coarse=nfc, smoother="gmres"))
    Ac = prob.AL[1].toarray()
    fc = prob.free[1]
    ec = np.zeros(g.coarse().N, dtype=complex)
    ec[fc] = np.linalg.solve(Ac[np.ix_(fc, fc)], (prob.P[0].T @ b)[fc])
    ref = prob.P[0] @ ec
    assert np.linalg.norm(prob.vcycle(0, b) - ref) <= 1e-9 * np.linalg.norm(ref)
    prob2 = O.Problem(g, 6.0, 0.0, 3.0, O.Options(levels=2, nu_pre=3, nu_post=2, nu_coarse=4, smoother="gmres",
                                                   gamma=2))
    c = 0.7 - 2.1j
    x = prob2.vcycle(0, b)
    assert np.linalg.norm(prob2.vcycle(0, c * b) - c * x) <= 1e-12 * abs(c) * np.linalg.norm(x)


def test_gmres_smoother_keeps_outer_counts_flat_in_k():
    """Sec. 5.3's multigrid (W-cycles, GMRES(5) with Jacobi on every level) at delta_hat = 2
    keeps the outer FGMRES counts nearly k-independent (10+ points per wavelength), while
    W(2,2) with damped Jacobi lets them grow: the reason the paper smooths with GMRES."""
    gm, jac = {}, {}
    for k, n in ((4.0, 16), (8.0, 32), (16.0, 64)):
        g = O.Grid(2, n, (S,) * 4)
        f = O.load_vector_nodal(g, inputs.gaussian_source(2, n, (0.4, 0.4), 0.05))
        for name, o in (("gmres", O.Options(levels=3, nu_pre=5, nu_post=5, nu_coarse=5, gamma=2, smoother="gmres")),
                        ("jacobi", O.Options(levels=3, gamma=2))):
            _, its, rel, _ = O.solve(O.Problem(g, k, 0.0, 2.0, o), f, 1e-8)
            assert rel <= 1e-8
            (gm if name == "gmres" else jac)[k] = its
    assert max(gm.values()) - min(gm.values()) <= 5, gm
    assert gm[16.0] < jac[16.0] and jac[16.0] - jac[4.0] > gm[16.0] - gm[4.0], (gm, jac)
