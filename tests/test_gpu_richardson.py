"""The preconditioned Richardson outer iteration (the stationary iteration after Def. 4.1)
on the GPU against the oracle's: same number of iterations, the same residual history to
rounding, and the LU solution at convergence."""
import numpy as np
import pytest
import torch

from oracle import hh_oracle as O
from nodewise import rel
from paper_2506_18694_gb300 import hh, inputs

pytestmark = pytest.mark.gpu

S, D = O.SOMMERFELD, O.DIRICHLET


@pytest.mark.parametrize("prec", [hh.HH_C128, hh.HH_C64])
@pytest.mark.parametrize("n,k,dh,cycles,bc", [
    (32, 10.0, 2.0, 1, (S, S, S, S)),
    (64, 20.0, 2.0, 2, (S, S, S, S)),
    (32, 10.0, 2.0, 2, (D, S, S, S)),
    (32, 12.0, 2.0, 1, (S, S, D, S)),
])
def test_richardson_matches_oracle(libhh, prec, n, k, dh, cycles, bc):
    g = O.Grid(2, n, bc)
    f = inputs.gaussian_source(2, n, (0.4, 0.6), 0.05)
    b = O.load_vector_nodal(g, f)
    oopts = O.Options(levels=3, cycles_per_hss=cycles, max_outer=300)
    prob = O.Problem(g, k, 0.0, dh, oopts)
    xo, its_o, rel_o, _ = O.solve_richardson(prob, b, 1e-8)
    assert rel_o <= 1e-8
    opts = hh.default_options(levels=3, cycles_per_hss=cycles, precision=prec, outer=hh.HH_OUTER_RICHARDSON,
                              max_outer=300)
    with hh.Problem(2, n, k, 0.0, dh, bc, opts) as p:
        u, info = p.solve(torch.from_numpy(b).cuda(), 1e-8)
        u = u.cpu().numpy()
    assert info.rel_residual <= 1e-8
    assert abs(info.outer_its - its_o) <= (0 if prec == hh.HH_C128 else 2)
    assert info.hss_its == info.outer_its * O.n_hss(k, 1.0)
    ref = prob.lu("B")(b)
    assert rel(u, ref) <= 1e-6
    res = np.linalg.norm(b - prob.B @ u) / np.linalg.norm(b)
    assert res <= 1.01e-8


def test_richardson_batch_equals_solo(libhh):
    g = O.Grid(2, 32, (S, S, S, S))
    ks = [10.0, 12.0, 10.0]
    f = np.concatenate([inputs.random_complex(g.N, 1600 + i) * g.free() for i in range(3)])
    opts = dict(levels=3, outer=hh.HH_OUTER_RICHARDSON, max_outer=300)
    with hh.Problem(2, 32, np.array(ks), 0.0, 2.0, (S, S, S, S), hh.default_options(**opts)) as pb:
        ub, infos = pb.solve(torch.from_numpy(f).cuda(), 1e-8)
        ub = ub.cpu().numpy().reshape(3, g.N)
    for i, k in enumerate(ks):
        with hh.Problem(2, 32, k, 0.0, 2.0, (S, S, S, S), hh.default_options(**opts)) as p:
            u, info = p.solve(torch.from_numpy(f[i * g.N:(i + 1) * g.N]).cuda(), 1e-8)
        assert np.array_equal(ub[i], u.cpu().numpy()) and infos[i].outer_its == info.outer_its


@pytest.mark.parametrize("outer", [hh.HH_OUTER_FGMRES, hh.HH_OUTER_RICHARDSON])
def test_theta_sweep_matches_oracle(libhh, outer):
    """ceil(k^theta) HSS steps per preconditioning for theta in {1/2, 1, 3/2} (Sec. 5.2):
    the GPU path takes the oracle's number of outer iterations (complex128 V-cycles)."""
    n, k, dh, bc = 32, 10.0, 2.0, (S, S, S, S)
    g = O.Grid(2, n, bc)
    b = O.load_vector_nodal(g, inputs.gaussian_source(2, n, (0.4, 0.6), 0.05))
    counts = []
    for theta in (0.5, 1.0, 1.5):
        prob = O.Problem(g, k, 0.0, dh, O.Options(levels=3, theta=theta, max_outer=300))
        solver = O.solve if outer == hh.HH_OUTER_FGMRES else O.solve_richardson
        _, its_o, rel_o, _ = solver(prob, b, 1e-8)
        opts = hh.default_options(levels=3, theta=theta, precision=hh.HH_C128, outer=outer, max_outer=300)
        with hh.Problem(2, n, k, 0.0, dh, bc, opts) as p:
            _, info = p.solve(torch.from_numpy(b).cuda(), 1e-8)
        assert info.outer_its == its_o and info.hss_its == its_o * O.n_hss(k, theta)
        if rel_o <= 1e-8:
            assert info.rel_residual <= 1e-8
        counts.append(its_o)
    assert counts[0] >= counts[1] >= counts[2]  # more HSS steps, fewer outer iterations
