"""Pins of the mixed-formulation oracle (oracle/hh_mixed.py) against facts other than itself:
the embedding property (the V_h mass and coupling reproduce the Q1 stiffness exactly), the
gradient of a bilinear function, the equivalence of the mixed and primal solutions that the
paper derives by eliminating sigma (Sec. 2), the elimination of sigma inside an HSS step
(Sec. 3.2), the H_mixed contraction of Prop. 3.6 at every step, and preconditioned FGMRES
against the primal sparse LU."""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

from oracle import hh_mixed as X
from oracle import hh_oracle as O
from paper_2506_18694_gb300 import inputs

S, D = O.SOMMERFELD, O.DIRICHLET


def _rand(n, seed):
    rng = np.random.default_rng(seed)
    return rng.standard_normal(n) + 1j * rng.standard_normal(n)


@pytest.mark.parametrize("dim,n,bc", [(2, 8, (S, D, S, S)), (2, 6, (D, D, D, D)), (3, 4, (S, S, S, S, D, S))])
def test_embedding_property_reproduces_stiffness(dim, n, bc):
    """grad Q_h lies in V_h, so G^T Ms^{-1} G is the Q1 stiffness matrix; Ms is SPD."""
    g = O.Grid(dim, n, bc)
    K, _, _ = O.assemble(g)
    Ms, G = X.assemble_mixed(g)
    schur = (G.T @ spla.spsolve(Ms.tocsc(), G.tocsc())).toarray()
    assert np.abs(schur - K.toarray()).max() <= 1e-12 * np.abs(K.toarray()).max()
    msd = Ms.toarray()
    assert np.allclose(msd, msd.T) and np.linalg.eigvalsh(msd).min() > 0


def test_gradient_of_bilinear_function():
    """For u = x y (in Q1), Ms^{-1} G u holds grad u exactly: sigma_x = y at the cell's two
    y-vertices, sigma_y = x at its two x-vertices."""
    g = O.Grid(2, 5, (S,) * 4)
    xy = g.coords()
    u = xy[:, 0] * xy[:, 1]
    Ms, G = X.assemble_mixed(g)
    sig = spla.spsolve(Ms.tocsc(), G @ u).reshape(g.n * g.n, 2, 2)
    h = g.h
    for c in range(g.n * g.n):
        i, j = c % g.n, c // g.n
        assert np.allclose(sig[c, 0], [j * h, (j + 1) * h], atol=1e-13)  # d/dx (xy) = y
        assert np.allclose(sig[c, 1], [i * h, (i + 1) * h], atol=1e-13)  # d/dy (xy) = x


@pytest.mark.parametrize("delta", [0.0, 0.5])
@pytest.mark.parametrize("dim,n,bc", [(2, 8, (S, S, D, S)), (3, 4, (S, S, S, S, D, S))])
def test_mixed_solution_is_primal_solution(dim, n, bc, delta):
    """Eliminating sigma recovers the primal formulation (Sec. 2): the mixed u solves
    B_delta u = M f, and sigma = grad u / (delta - i k)."""
    g = O.Grid(dim, n, bc)
    k = 5.0
    p = X.MixedProblem(g, k, delta, k)
    f = inputs.random_complex(g.N, 40 + n) * g.free()
    U = p.lu_solve(p.rhs(f))
    sig, u = p.split(U)
    prim = O.Problem(g, k, delta, k, O.Options(levels=1))
    ref = prim.lu("B")(prim.mats[0][1] @ f)
    assert np.linalg.norm(u - ref) <= 1e-10 * np.linalg.norm(ref)
    grad = spla.spsolve(p.Ms.tocsc(), p.G @ u)
    assert np.linalg.norm(sig - grad / (delta - 1j * k)) <= 1e-10 * np.linalg.norm(sig)


@pytest.mark.parametrize("dim,n,bc", [(2, 8, (S, D, S, S)), (3, 4, (S, S, D, S, S, S))])
def test_hss_step_elimination_equals_block_solve(dim, n, bc):
    """Def. 4.2's step solved as the 2 x 2 block system and through the eliminated
    u-equation A_mix u' = k (dh - i) g_u - G^T Ms^{-1} g_s agree."""
    g = O.Grid(dim, n, bc)
    p = X.MixedProblem(g, 7.0, 0.0, 2.0)
    U = _rand(p.ns + p.N, 50) * p.free
    R = _rand(p.ns + p.N, 51) * p.free
    a = p.hss_step_direct(U, R)
    b = p.hss_step_eliminated(U, R)
    assert np.linalg.norm(a - b) <= 1e-10 * np.linalg.norm(a)


@pytest.mark.parametrize("dim,k,dh", [(2, 6.0, 1.0), (2, 12.0, 0.3), (3, 5.0, 0.5)])
def test_mixed_hss_contracts_in_h_norm(dim, k, dh):
    """Prop. 3.6: for the shifted mixed system (delta = dh > 0) each HSS step contracts the
    error by (k - 1)/(k + 1) or better in the H_mixed norm."""
    g = O.Grid(dim, 8 if dim == 2 else 4, (S, S, S, D) if dim == 2 else (S, S, S, S, D, S))
    p = X.MixedProblem(g, k, dh, dh)
    F = p.rhs(inputs.random_complex(g.N, 60) * g.free())
    Ustar = p.lu_solve(F)
    H = p.H(dh)
    hnorm = lambda e: np.sqrt(np.real(np.vdot(e, H @ e)))
    U = np.zeros_like(Ustar)
    rate = (k - 1) / (k + 1)
    e = hnorm(U - Ustar)
    for _ in range(12):
        U = p.hss_step_direct(U, F, dh)
        e1 = hnorm(U - Ustar)
        assert e1 <= rate * e * (1 + 1e-9)
        e = e1


def test_mixed_fgmres_matches_primal_lu():
    """FGMRES on the mixed system (delta = 0) with the shifted-HSS preconditioner of Def. 4.2:
    with exact u-solves and with multigrid cycles on A_mix, the u it returns is the primal
    sparse-LU solution."""
    g = O.Grid(2, 16, (S,) * 4)
    k = 6.0
    f = O.load_vector_nodal(g, inputs.gaussian_source(2, 16, (0.4, 0.4), 0.05))
    prim = O.Problem(g, k, 0.0, k, O.Options(levels=1))
    ref = prim.lu("B")(f)
    fn = spla.spsolve(prim.mats[0][1].tocsc(), f)  # nodal source whose load vector is f
    for inner, tol in ((None, 1e-10), ("mg", 1e-8)):
        p = X.MixedProblem(g, k, 0.0, k, O.Options(levels=3))
        b = p.rhs(fn)
        U, its, rel, _ = p.solve(b, tol, inner=inner)
        _, u = p.split(U)
        assert rel <= tol and its <= 60
        assert np.linalg.norm(u - ref) <= 1e-6 * np.linalg.norm(ref)


def test_mixed_outer_counts_follow_primal():
    """After the elimination of sigma the mixed preconditioner solves a primal-type shifted
    problem (Sec. 3.2), so with the same multigrid (4 levels, V(2,2)-Jacobi) the outer FGMRES
    counts of the two formulations stay within a few iterations of each other, both
    k-independent at delta_hat = 2."""
    g = O.Grid(2, 32, (S,) * 4)
    f = O.load_vector_nodal(g, inputs.gaussian_source(2, 32, (0.4, 0.4), 0.05))
    counts = {}
    for k in (6.0, 12.0):
        prim = O.Problem(g, k, 0.0, 2.0, O.Options(levels=4))
        _, its_p, rel_p, _ = O.solve(prim, f, 1e-8)
        fn = spla.spsolve(prim.mats[0][1].tocsc(), f)
        xp = X.MixedProblem(g, k, 0.0, 2.0, O.Options(levels=4))
        _, its_m, rel_m, _ = xp.solve(xp.rhs(fn), 1e-8)
        assert rel_p <= 1e-8 and rel_m <= 1e-8
        assert abs(its_m - its_p) <= 3, (k, its_m, its_p)
        counts[k] = its_m
    assert counts[12.0] <= counts[6.0] + 3
