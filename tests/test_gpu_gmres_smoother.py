"""GMRES smoother with a Jacobi preconditioner (Sec. 5.3: GMRES iterations on every level,
the coarsest included, inside W-cycles) on the GPU against the oracle.

The GPU orthogonalises by classical Gram-Schmidt twice and solves the small least-squares
problem by Givens rotations; the oracle uses modified Gram-Schmidt and a dense least-squares
solve, so the two agree to rounding: 1e-10 relative in complex128 (a few levels of s <= 5
iterations, each a well-conditioned 6 x 5 least-squares problem) and 2e-4 in complex64 (FP32
basis vectors and block sums; the block shares combined in FP64).  Solves are checked against
sparse LU; batches and graph replays must equal lone, eager runs bit for bit (fixed-order
sums).
"""
import numpy as np
import pytest
import torch

from oracle import hh_oracle as O
from nodewise import rel
from paper_2506_18694_gb300 import hh, inputs

pytestmark = pytest.mark.gpu

S, D = O.SOMMERFELD, O.DIRICHLET
TOL = {hh.HH_C128: 1e-10, hh.HH_C64: 2e-4}
DT = {hh.HH_C128: torch.complex128, hh.HH_C64: torch.complex64}
GM = hh.HH_SMOOTH_GMRES


def _opts(levels, nu, gamma):
    return dict(levels=levels, nu_pre=nu[0], nu_post=nu[1], nu_coarse=nu[2], cycle_gamma=gamma)


@pytest.mark.parametrize("prec", [hh.HH_C128, hh.HH_C64])
@pytest.mark.parametrize("dim,n,levels,bc,nu,gamma", [
    (2, 32, 3, (S, S, S, S), (5, 5, 5), 2),
    (2, 40, 4, (D, S, S, D), (3, 2, 4), 1),
    (2, 64, 4, (S, D, S, S), (1, 0, 8), 2),
    (3, 16, 3, (S, S, S, S, D, S), (4, 4, 4), 2),
], ids=["2d-w55", "2d-v324", "2d-w108", "3d-w444"])
def test_gmres_cycle_matches_oracle(libhh, prec, dim, n, levels, bc, nu, gamma):
    g = O.Grid(dim, n, bc)
    o = _opts(levels, nu, gamma)
    prob = O.Problem(g, 7.0, 0.0, 2.5, O.Options(smoother="gmres", gamma=gamma,
                                                 **{k: v for k, v in o.items() if k != "cycle_gamma"}))
    b = inputs.random_complex(g.N, 2100 + n) * g.free()
    ref = prob.vcycle(0, b)
    with hh.Problem(dim, n, 7.0, 0.0, 2.5, bc, hh.default_options(precision=prec, smoother=GM, **o)) as p:
        x = p.vcycle(torch.from_numpy(b).to(DT[prec]).cuda()).cpu().numpy().astype(np.complex128)
    assert rel(x, ref) <= TOL[prec]


@pytest.mark.parametrize("prec", [hh.HH_C128, hh.HH_C64])
def test_gmres_preconditioner_matches_oracle(libhh, prec):
    """The HSS loop of Def. 4.1 with W-cycles and GMRES(3) smoothing, two cycles per step."""
    g = O.Grid(2, 32, (S, S, D, S))
    o = dict(levels=3, nu_pre=3, nu_post=3, nu_coarse=3, cycles_per_hss=2)
    prob = O.Problem(g, 6.0, 0.0, 2.0, O.Options(smoother="gmres", gamma=2, **o))
    r = inputs.random_complex(g.N, 2200) * g.free()
    ref = prob.prec(r)
    with hh.Problem(2, 32, 6.0, 0.0, 2.0, g.bc, hh.default_options(precision=prec, smoother=GM, cycle_gamma=2,
                                                                   **o)) as p:
        z = p.precondition(torch.from_numpy(r).cuda()).cpu().numpy()
    assert rel(z, ref) <= 10 * TOL[prec]


@pytest.mark.parametrize("dim,n,k,bc", [(2, 64, 16.0, (S, S, S, S)), (3, 16, 6.0, (S, S, S, S, D, S))])
def test_gmres_smoothed_solve_against_lu(libhh, dim, n, k, bc):
    """Paper settings (W-cycle, GMRES(5) on every level) at delta_hat = 2: the solve reaches
    the tolerance, matches sparse LU, and takes the oracle's outer iteration count (FP64
    cycles; the complex64 solve within two iterations of it)."""
    g = O.Grid(dim, n, bc)
    o = dict(levels=3, nu_pre=5, nu_post=5, nu_coarse=5)
    prob = O.Problem(g, k, 0.0, 2.0, O.Options(smoother="gmres", gamma=2, **o))
    b = O.load_vector_nodal(g, inputs.gaussian_source(dim, n, (0.4,) * dim, 0.05))
    _, its_ref, _, _ = O.solve(prob, b, 1e-8)
    ref = prob.lu("B")(b)
    for prec in (hh.HH_C128, hh.HH_C64):
        with hh.Problem(dim, n, k, 0.0, 2.0, bc, hh.default_options(precision=prec, smoother=GM, cycle_gamma=2,
                                                                    **o)) as p:
            u, info = p.solve(torch.from_numpy(b).cuda(), 1e-8)
            u = u.cpu().numpy()
        assert info.rel_residual <= 1e-8
        assert rel(u, ref) <= 1e-6
        if prec == hh.HH_C128:
            assert info.outer_its == its_ref
        else:
            assert abs(info.outer_its - its_ref) <= 2


def test_gmres_batch_and_graphs_equal_lone_eager(libhh):
    g = O.Grid(2, 32, (S, S, S, D))
    mix = [(10.0, 0.0, 2.0), (6.0, 0.4, 3.0), (14.0, 0.0, 14.0)]
    o = dict(levels=3, nu_pre=4, nu_post=3, nu_coarse=5, cycle_gamma=2, smoother=GM)
    nb = len(mix)
    f = np.stack([inputs.random_complex(g.N, 2300 + q) * g.free() for q in range(nb)])
    ks, ds, dhs = (np.array(c) for c in zip(*mix))
    with hh.Problem(2, 32, ks, ds, dhs, g.bc, hh.default_options(**o)) as pb:
        ub, infos = pb.solve(torch.from_numpy(f.reshape(-1)).cuda(), 1e-8)
        ub = ub.cpu().numpy().reshape(nb, -1)
        vb = pb.vcycle(torch.from_numpy(f.reshape(-1)).to(torch.complex64).cuda()).cpu().numpy().reshape(nb, -1)
    for q, (k, d, dh) in enumerate(mix):
        for graphs in (1, 0):
            with hh.Problem(2, 32, k, d, dh, g.bc, hh.default_options(use_graphs=graphs, **o)) as p:
                u, info = p.solve(torch.from_numpy(f[q]).cuda(), 1e-8)
                assert np.array_equal(u.cpu().numpy(), ub[q]), (q, graphs)
                assert info.outer_its == infos[q].outer_its
                v = p.vcycle(torch.from_numpy(f[q]).to(torch.complex64).cuda()).cpu().numpy()
                assert np.array_equal(v, vb[q]), (q, graphs)


def test_gmres_device_bytes_match_footprint(libhh):
    o = hh.default_options(levels=3, nu_pre=5, nu_post=5, nu_coarse=5, cycle_gamma=2, smoother=GM)
    with hh.Problem(2, 64, np.array([8.0, 12.0]), np.zeros(2), np.array([2.0, 2.0]), (S,) * 4, o) as p:
        _, infos = p.solve(torch.ones(2 * 65 * 65, dtype=torch.complex128).cuda(), 1e-6)
    assert infos[0].device_bytes == hh.footprint_bytes(2, 64, o, nb=2)
    assert hh.footprint_bytes(2, 64, o, nb=2) > hh.footprint_bytes(2, 64, hh.default_options(
        levels=3, nu_pre=5, nu_post=5, nu_coarse=5, cycle_gamma=2), nb=2)
