"""W-cycles (cycle index 2, the paper's cycle type, Sec. 5.3) on the GPU against the oracle:
the cycle as an operator (complex128 1e-12, complex64 2e-5, as the V-cycle parity tests),
and solves against sparse LU."""
import numpy as np
import pytest
import torch

from oracle import hh_oracle as O
from nodewise import rel
from paper_2506_18694_gb300 import hh, inputs

pytestmark = pytest.mark.gpu

S, D = O.SOMMERFELD, O.DIRICHLET
TOL = {hh.HH_C128: 1e-12, hh.HH_C64: 2e-5}
DT = {hh.HH_C128: torch.complex128, hh.HH_C64: torch.complex64}


@pytest.mark.parametrize("prec", [hh.HH_C128, hh.HH_C64])
@pytest.mark.parametrize("dim,n,levels,bc,gamma", [
    (2, 72, 4, (S, S, S, S), 2),
    (2, 32, 3, (D, S, S, D), 3),
    (3, 16, 3, (S, S, S, S, D, S), 2),
])
def test_w_cycle_matches_oracle(libhh, prec, dim, n, levels, bc, gamma):
    g = O.Grid(dim, n, bc)
    prob = O.Problem(g, 7.0, 0.0, 2.5, O.Options(levels=levels, gamma=gamma))
    b = inputs.random_complex(g.N, 1700 + n) * g.free()
    ref = prob.vcycle(0, b)
    with hh.Problem(dim, n, 7.0, 0.0, 2.5, bc, hh.default_options(levels=levels, precision=prec,
                                                                  cycle_gamma=gamma)) as p:
        x = p.vcycle(torch.from_numpy(b).to(DT[prec]).cuda()).cpu().numpy().astype(np.complex128)
    assert rel(x, ref) <= TOL[prec]


@pytest.mark.parametrize("dim,n,bc", [(2, 64, (S, S, S, S)), (3, 16, (S, S, S, S, D, S))])
def test_w_cycle_solve_against_lu(libhh, dim, n, bc):
    g = O.Grid(dim, n, bc)
    k = 12.0 if dim == 2 else 6.0
    prob = O.Problem(g, k, 0.0, k, O.Options(levels=3))
    b = O.load_vector_nodal(g, inputs.gaussian_source(dim, n, (0.4,) * dim, 0.05))
    with hh.Problem(dim, n, k, 0.0, k, bc, hh.default_options(levels=3, cycle_gamma=2)) as p:
        u, info = p.solve(torch.from_numpy(b).cuda(), 1e-9)
        u = u.cpu().numpy()
    ref = prob.lu("B")(b)
    assert info.rel_residual <= 1e-9
    assert rel(u, ref) <= 1e-6
