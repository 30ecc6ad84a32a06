"""Mixed formulation on the GPU (Sec. 2, Def. 4.2) against the mixed oracle: the FP64 system
operator, the shifted-HSS preconditioner through the elimination of sigma (cycles on A_mix),
and solves against the primal sparse LU (eliminating sigma recovers the primal solution).

Tolerances: the system operator 1e-12 (the same sums in another order); the preconditioner
1e-10 with complex128 cycles and 1e-4 with complex64 ones (ceil(k) HSS steps of FP32 cycles);
solves reach the relative residual 1e-8 and the primal LU solution to 1e-6."""
import numpy as np
import pytest
import scipy.sparse.linalg as spla
import torch

from oracle import hh_mixed as X
from oracle import hh_oracle as O
from nodewise import rel
from paper_2506_18694_gb300 import hh, inputs

pytestmark = pytest.mark.gpu

S, D = O.SOMMERFELD, O.DIRICHLET
MIXED = hh.HH_FORM_MIXED


def _rand(n, seed):
    rng = np.random.default_rng(seed)
    return rng.standard_normal(n) + 1j * rng.standard_normal(n)


@pytest.mark.parametrize("dim,n,bc", [(2, 8, (S, D, S, S)), (2, 24, (S, S, S, S)), (3, 4, (S, S, S, S, D, S)),
                                      (3, 8, (D, S, S, S, S, S))])
def test_mixed_system_operator_matches_oracle(libhh, dim, n, bc):
    g = O.Grid(dim, n, bc)
    xp = X.MixedProblem(g, 6.0, 0.4, 3.0)
    assert hh.load_library().hh_sigma_dofs(hh.Grid(dim, n)) == xp.ns
    U = _rand(xp.ns + g.N, 70 + n) * xp.free
    with hh.Problem(dim, n, 6.0, 0.4, 3.0, bc, hh.default_options(levels=2, formulation=MIXED)) as p:
        assert p.system_size() == xp.ns + g.N
        y = p.apply_system(torch.from_numpy(U).cuda()).cpu().numpy()
    ref = xp.A() @ U
    assert rel(y, ref) <= 1e-12


@pytest.mark.parametrize("prec,tol", [(hh.HH_C128, 1e-10), (hh.HH_C64, 1e-4)])
@pytest.mark.parametrize("dim,n,levels,bc", [(2, 32, 3, (S, S, D, S)), (3, 8, 2, (S, S, S, S, D, S))])
def test_mixed_preconditioner_matches_oracle(libhh, prec, tol, dim, n, levels, bc):
    g = O.Grid(dim, n, bc)
    k, dh = 5.0, 2.0
    xp = X.MixedProblem(g, k, 0.0, dh, O.Options(levels=levels))
    R = _rand(xp.ns + g.N, 80 + n) * xp.free
    ref = xp.prec(R)
    with hh.Problem(dim, n, k, 0.0, dh, bc, hh.default_options(levels=levels, precision=prec,
                                                               formulation=MIXED)) as p:
        z = p.precondition(torch.from_numpy(R).cuda()).cpu().numpy()
    assert rel(z, ref) <= tol


@pytest.mark.parametrize("dim,n,k,dh,bc", [
    (2, 32, 6.0, 6.0, (S, S, S, S)),
    (2, 32, 12.0, 2.0, (S, S, D, S)),
    (3, 8, 4.0, 4.0, (S, S, S, S, D, S)),
])
def test_mixed_solve_matches_primal_lu(libhh, dim, n, k, dh, bc):
    g = O.Grid(dim, n, bc)
    levels = 3 if dim == 2 else 2
    f = inputs.gaussian_source(dim, n, (0.4,) * dim, 0.05) * g.free()
    xp = X.MixedProblem(g, k, 0.0, dh, O.Options(levels=levels))
    b = xp.rhs(f)
    _, its_ref, _, _ = xp.solve(b, 1e-8)
    prim = O.Problem(g, k, 0.0, k, O.Options(levels=1))
    uref = prim.lu("B")(prim.mats[0][1] @ f)
    sref = spla.spsolve(xp.Ms.tocsc(), xp.G @ uref) / (0.0 - 1j * k)
    for prec in (hh.HH_C128, hh.HH_C64):
        with hh.Problem(dim, n, k, 0.0, dh, bc, hh.default_options(levels=levels, precision=prec,
                                                                   formulation=MIXED)) as p:
            U, info = p.solve(torch.from_numpy(b).cuda(), 1e-8)
            U = U.cpu().numpy()
        sig, u = U[:xp.ns], U[xp.ns:]
        assert info.rel_residual <= 1e-8
        assert rel(u, uref) <= 1e-6
        assert rel(sig, sref) <= 1e-6
        if prec == hh.HH_C128:
            assert info.outer_its == its_ref
        else:
            assert abs(info.outer_its - its_ref) <= 2
