"""Pins of the plain-C OpenMP oracle (oracle/hss_omp.c) against facts other than itself.

The C oracle restates the V-cycle, the shifted-HSS preconditioner of Def. 4.1 and FGMRES
(Sec. 5.1) for grids too large for the Python oracle.  It is checked here against the dense
error-propagation formula of a multigrid cycle, the power of that formula for several
cycles per HSS step, the pinned Python oracle step for step, and sparse LU.
"""
import numpy as np
import pytest

from oracle import hh_oracle as O
from oracle import hss_omp as C
from test_oracle_pins import _dense_vcycle_operator

S, D = O.SOMMERFELD, O.DIRICHLET


def _rand(n, seed):
    rng = np.random.default_rng(seed)
    return rng.standard_normal(n) + 1j * rng.standard_normal(n)


@pytest.mark.parametrize("bc", [(S, S, S, S), (D, S, S, D)])
def test_c_vcycle_matches_error_propagation_formula(bc):
    g = O.Grid(2, 8, bc)
    prob = O.Problem(g, 5.0, 0.0, 2.0, O.Options(levels=3, nu_pre=1, nu_post=2, nu_coarse=3))
    B = _dense_vcycle_operator(prob, 0)
    b = _rand(g.N, 5) * g.free()
    x = C.COracle(prob).vcycle(0, b)
    assert np.abs(x - B @ b).max() <= 1e-11 * np.abs(B @ b).max()
    assert np.all(x[~g.free()] == 0)


@pytest.mark.parametrize("cycles", [2, 3])
def test_c_mg_solve_cycles_match_error_propagation_power(cycles):
    g = O.Grid(2, 8, (D, S, S, D))
    prob = O.Problem(g, 5.0, 0.0, 2.0, O.Options(levels=3, nu_pre=1, nu_post=2, nu_coarse=3,
                                                 cycles_per_hss=cycles))
    B = _dense_vcycle_operator(prob, 0)
    A = prob.AL[0].toarray()
    f = prob.free[0]
    b = _rand(g.N, 6) * g.free()
    xe = np.zeros(g.N, dtype=complex)
    xe[f] = np.linalg.solve(A[np.ix_(f, f)], b[f])
    want = xe - np.linalg.matrix_power(np.eye(g.N) - B @ A, cycles) @ xe
    got = C.COracle(prob).mg_solve(b)
    assert np.abs(got - want).max() <= 1e-10 * np.abs(want).max()


@pytest.mark.parametrize("dim,n,L,bc,cycles", [
    (2, 32, 4, (S, S, S, S), 1),
    (2, 24, 3, (D, S, S, D), 2),
    (3, 8, 3, (S, S, S, S, D, S), 1),
])
def test_c_preconditioner_equals_python_oracle(dim, n, L, bc, cycles):
    g = O.Grid(dim, n, bc)
    prob = O.Problem(g, 6.0, 0.0, 6.0, O.Options(levels=L, cycles_per_hss=cycles))
    r = _rand(g.N, 7) * g.free()
    want = prob.prec(r)
    got = C.COracle(prob).prec(r)
    assert np.abs(got - want).max() <= 1e-12 * np.abs(want).max()


@pytest.mark.parametrize("dim,n,k,dh,bc", [
    (2, 32, 10.0, 10.0, (S, S, S, S)),
    (2, 32, 8.0, 2.0, (D, S, S, D)),
    (3, 16, 6.0, 6.0, (S, S, S, S, D, S)),
])
def test_c_fgmres_matches_lu(dim, n, k, dh, bc):
    g = O.Grid(dim, n, bc)
    prob = O.Problem(g, k, 0.0, dh, O.Options(levels=3, cycles_per_hss=2 if dh == 2.0 else 1))
    b = O.load_vector_nodal(g, np.exp(-((g.coords() - 0.4) ** 2).sum(axis=1) / (2 * 0.05 ** 2)))
    x, its, rr = C.COracle(prob).fgmres(b, 1e-10, restart=30, max_it=300)
    assert rr <= 1e-10
    assert np.linalg.norm(b - prob.B @ x) <= 1.01e-10 * np.linalg.norm(b)
    ex = prob.lu("B")(b)
    assert np.linalg.norm(x - ex) <= 1e-7 * np.linalg.norm(ex)
    assert np.all(x[~g.free()] == 0)


def test_c_thread_count_does_not_change_the_cycle():
    g = O.Grid(2, 64, (S, S, S, S))
    prob = O.Problem(g, 10.0, 0.0, 10.0, O.Options())
    c = C.COracle(prob)
    r = _rand(g.N, 8)
    saved = C.COracle.threads()
    try:
        C.COracle.threads(1)
        a = c.mg_solve(r)
        C.COracle.threads(4)
        b = c.mg_solve(r)
    finally:
        C.COracle.threads(saved)
    assert np.array_equal(a, b)  # row-parallel products: the same sums in the same order
