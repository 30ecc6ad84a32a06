"""Batches of problems: one hh_problem holding nb problems (their own k, delta, delta_hat and
HSS lengths) runs every kernel over all of them at once.  Each problem's result must be the
one a batch of one gives, bit for bit: the same kernels with the same per-problem arithmetic,
a problem whose HSS loop or outer iteration has ended being skipped, never recomputed.  The
batched solves are also checked against the oracle's sparse LU.
"""
import numpy as np
import pytest
import torch

from oracle import hh_oracle as O
from nodewise import rel
from paper_2506_18694_gb300 import hh, inputs

pytestmark = pytest.mark.gpu

S, D = O.SOMMERFELD, O.DIRICHLET

# (k, delta, delta_hat): HSS lengths 10, 20, 20, 30 (ceil(k^theta), theta = 1)
MIX = [(10.0, 0.0, 10.0), (20.0, 0.0, 20.0), (20.0, 0.5, 2.0), (30.0, 0.0, 30.0)]


def _batch(dim, n, bc, mix, **opt):
    ks, ds, dhs = (np.array(c) for c in zip(*mix))
    return hh.Problem(dim, n, ks, ds, dhs, bc, hh.default_options(**opt))


def _rhs(g, nb, seed):
    return np.stack([inputs.random_complex(g.N, seed + b) * g.free() for b in range(nb)])


@pytest.mark.parametrize("dim,n,bc,opt", [
    (2, 64, (S, S, S, S), dict(levels=3)),
    (2, 64, (D, S, S, D), dict(levels=3, precision=hh.HH_C128)),
    (2, 64, (S, S, S, S), dict(levels=3, use_graphs=0, nu_pre=0, nu_post=1)),
    (2, 64, (S, S, S, S), dict(levels=3, cycles_per_hss=2, restart=5)),
    (3, 16, (S, S, S, S, D, S), dict(levels=3)),
], ids=["2d", "2d-dir-c128", "2d-nopre-nographs", "2d-2cycles-restart5", "3d"])
def test_batched_solve_equals_solo(libhh, dim, n, bc, opt):
    g = O.Grid(dim, n, bc)
    nb = len(MIX)
    f = _rhs(g, nb, 500)
    with _batch(dim, n, bc, MIX, **opt) as pb:
        ub, infos = pb.solve(torch.from_numpy(f.reshape(-1)).cuda(), 1e-9)
        ub = ub.cpu().numpy().reshape(nb, g.N)
    assert len(infos) == nb
    for b, (k, delta, dh) in enumerate(MIX):
        with hh.Problem(dim, n, k, delta, dh, bc, hh.default_options(**opt)) as p:
            u, info = p.solve(torch.from_numpy(f[b]).cuda(), 1e-9)
            u = u.cpu().numpy()
        assert np.array_equal(ub[b], u), b
        assert infos[b].outer_its == info.outer_its and infos[b].hss_its == info.hss_its
        assert infos[b].rel_residual == info.rel_residual and info.rel_residual <= 1e-9
        assert infos[b].hss_its == info.outer_its * O.n_hss(k, 1.0)


def test_batched_solve_against_lu(libhh):
    dim, n, bc = 2, 32, (S, S, D, S)
    g = O.Grid(dim, n, bc)
    nb = len(MIX)
    f = _rhs(g, nb, 600)
    with _batch(dim, n, bc, MIX, levels=3) as pb:
        u, infos = pb.solve(torch.from_numpy(f.reshape(-1)).cuda(), 1e-10)
        u = u.cpu().numpy().reshape(nb, g.N)
    for b, (k, delta, dh) in enumerate(MIX):
        prob = O.Problem(g, k, delta, dh, O.Options(levels=1))
        ref = prob.lu("B")(f[b] * g.free())
        assert rel(u[b], ref) <= 1e-7, b
        assert infos[b].rel_residual <= 1e-10


def test_batched_host_solve_and_zero_member(libhh):
    """solve_host over a batch; a zero right side in the batch gives u = 0 exactly."""
    dim, n, bc = 2, 32, (S, S, S, S)
    g = O.Grid(dim, n, bc)
    f = _rhs(g, 3, 700)
    f[1] = 0.0
    mix = MIX[:3]
    with _batch(dim, n, bc, mix, levels=3) as pb:
        u, infos = pb.solve_host(f.reshape(-1), 1e-9)
        ud, _ = pb.solve(torch.from_numpy(f.reshape(-1)).cuda(), 1e-9)
    u = u.reshape(3, g.N)
    assert np.all(u[1] == 0) and infos[1].outer_its == 0
    assert np.array_equal(u, ud.cpu().numpy().reshape(3, g.N))
    assert infos[0].rel_residual <= 1e-9 and infos[2].rel_residual <= 1e-9


@pytest.mark.parametrize("prec", [hh.HH_C128, hh.HH_C64])
@pytest.mark.parametrize("dim,n,bc,form", [
    (2, 72, (S, S, D, S), 0), (2, 72, (S, S, D, S), 1), (2, 72, (S, S, D, S), 2), (3, 12, (S, S, S, S, S, D), 0),
], ids=["2d", "2d-tile", "2d-persistent", "3d"])
def test_batched_building_blocks_equal_solo(libhh, prec, dim, n, bc, form):
    """Batched kernels against batches of one; the batch runs the tile form `form`
    (persistent warps walk every problem's tiles), the problems of one the automatic form.
    The coarse output of the residual restriction sits in a larger buffer whose tail must
    stay untouched."""
    dt = torch.complex128 if prec == hh.HH_C128 else torch.complex64
    g = O.Grid(dim, n, bc)
    nb = len(MIX)
    L = 3
    x = _rhs(g, nb, 800)
    r = _rhs(g, nb, 900)
    gc = O.Grid(dim, n // 2, bc)
    ec = np.stack([inputs.random_complex(gc.N, 950 + b) for b in range(nb)])
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a.reshape(-1))).to(dt).cuda()
    nc = nb * gc.N
    guarded = torch.full((nc * 16,), complex(7.0, -3.0), dtype=dt).cuda()
    with _batch(dim, n, bc, MIX, levels=L, precision=prec, tile_form=form) as pb:
        out_b = {
            "AL": pb.apply(0, "AL", dev(x)), "B": pb.apply(1, "B", dev(ec)),
            "jac": pb.jacobi(0, dev(r), dev(x)), "jac0": pb.jacobi(0, dev(r)),
            "rr": pb.residual_restrict(0, dev(r), dev(x), guarded[:nc]), "pc": pb.prolong_correct(0, dev(ec), dev(x)),
            "vc": pb.vcycle(dev(r)), "hr": pb.hss_rhs(dev(x), dev(r)),
        }
        assert bool((guarded[nc:] == complex(7.0, -3.0)).all()), "write past the coarse output"
        out_b = {k: v.cpu().numpy().reshape(nb, -1) for k, v in out_b.items()}
        xd, rd = (torch.from_numpy(a.reshape(-1)).cuda() for a in (x, r))
        dots = pb.dot(xd, rd)
        pre = pb.precondition(rd).cpu().numpy().reshape(nb, -1)
    for b, (k, delta, dh) in enumerate(MIX):
        with hh.Problem(dim, n, k, delta, dh, bc, hh.default_options(levels=L, precision=prec)) as p:
            one = {
                "AL": p.apply(0, "AL", dev(x[b])), "B": p.apply(1, "B", dev(ec[b])),
                "jac": p.jacobi(0, dev(r[b]), dev(x[b])), "jac0": p.jacobi(0, dev(r[b])),
                "rr": p.residual_restrict(0, dev(r[b]), dev(x[b])), "pc": p.prolong_correct(0, dev(ec[b]), dev(x[b])),
                "vc": p.vcycle(dev(r[b])), "hr": p.hss_rhs(dev(x[b]), dev(r[b])),
            }
            for key, v in one.items():
                assert np.array_equal(out_b[key][b], v.cpu().numpy()), (key, b)
            xb, rb = torch.from_numpy(x[b]).cuda(), torch.from_numpy(r[b]).cuda()
            assert dots[b] == p.dot(xb, rb)
            assert np.array_equal(pre[b], p.precondition(rb).cpu().numpy()), b
        assert abs(dots[b] - np.vdot(x[b], r[b])) <= 1e-12 * np.linalg.norm(x[b]) * np.linalg.norm(r[b])


def test_batch_device_bytes_match_footprint(libhh):
    dim, n, bc = 2, 64, (S, S, S, S)
    g = O.Grid(dim, n, bc)
    opts = dict(levels=3, restart=10)
    with _batch(dim, n, bc, MIX, **opts) as pb:
        _, infos = pb.solve(torch.from_numpy(_rhs(g, len(MIX), 1000).reshape(-1)).cuda(), 1e-6)
    assert infos[0].device_bytes == hh.footprint_bytes(dim, n, hh.default_options(**opts), nb=len(MIX))


def test_binding_rejects_wrong_sizes(libhh):
    with _batch(2, 32, (S, S, S, S), MIX, levels=3) as pb:
        short = torch.zeros(pb.nodes(0), dtype=torch.complex128, device="cuda")
        with pytest.raises(ValueError):
            pb.solve(short)
        with pytest.raises(ValueError):
            pb.apply(0, "AL", short)


def test_large_batch_coarse_clusters_equal_solo(libhh):
    """24 problems: the coarsest-level solve runs smaller clusters per problem than a batch
    of one does (so that all clusters are resident at once); results stay bit for bit."""
    dim, n, bc = 2, 64, (S, D, S, S)
    g = O.Grid(dim, n, bc)
    mix = [MIX[i % len(MIX)] for i in range(24)]
    f = _rhs(g, len(mix), 1200)
    with _batch(dim, n, bc, mix, levels=3) as pb:
        ub, infos = pb.solve(torch.from_numpy(f.reshape(-1)).cuda(), 1e-9)
        ub = ub.cpu().numpy().reshape(len(mix), g.N)
    for b in (0, 5, 11, 23):
        k, delta, dh = mix[b]
        with hh.Problem(dim, n, k, delta, dh, bc, hh.default_options(levels=3)) as p:
            u, info = p.solve(torch.from_numpy(f[b]).cuda(), 1e-9)
        assert np.array_equal(ub[b], u.cpu().numpy()), b
        assert infos[b].outer_its == info.outer_its
