"""Fused two-sweep kernels (2D): the HSS right side with the first two pre-sweeps and the
prolongation with the first two post-sweeps run as one pass.  Each node's arithmetic is the
one-sweep kernels', so V-cycles, preconditioner applications and solves must equal the
unfused path bit for bit (and the oracle, through the parity tests that run fused by default)."""
import numpy as np
import pytest
import torch

from oracle import hh_oracle as O
from paper_2506_18694_gb300 import hh, inputs

pytestmark = pytest.mark.gpu

S, D = O.SOMMERFELD, O.DIRICHLET


@pytest.mark.parametrize("prec", [hh.HH_C64, hh.HH_C128])
@pytest.mark.parametrize("n,levels,bc,nu", [
    (72, 4, (S, S, S, S), (2, 2)),
    (64, 3, (D, S, S, D), (2, 2)),
    (40, 3, (S, D, D, S), (3, 3)),
    (16, 1, (S, S, S, S), (2, 2)),
    (128, 4, (S, S, D, S), (2, 1)),
])
def test_fused_equals_unfused(libhh, prec, n, levels, bc, nu):
    g = O.Grid(2, n, bc)
    dt = torch.complex64 if prec == hh.HH_C64 else torch.complex128
    r = torch.from_numpy(inputs.random_complex(g.N, 1300 + n) * g.free()).cuda()
    out = {}
    for fuse in (0, 1):
        opts = hh.default_options(levels=levels, precision=prec, nu_pre=nu[0], nu_post=nu[1], fuse_sweeps=fuse)
        with hh.Problem(2, n, 15.0, 0.0, 15.0, bc, opts) as p:
            v = p.vcycle(r.to(dt))
            z = p.precondition(r)
            u, info = p.solve(r, 1e-9)
            out[fuse] = (v.cpu(), z.cpu(), u.cpu(), info.outer_its)
    for q in range(3):
        d = float((out[0][q] - out[1][q]).abs().max() / out[0][q].abs().max())
        assert torch.equal(out[0][q], out[1][q]), (q, d)
    assert torch.equal(out[0][2], out[1][2]) and out[0][3] == out[1][3]


def test_fused_batch_equals_unfused(libhh):
    n, bc = 64, (S, S, S, D)
    g = O.Grid(2, n, bc)
    ks = np.array([10.0, 20.0, 30.0])
    f = torch.from_numpy(np.concatenate([inputs.random_complex(g.N, 1400 + b) * g.free() for b in range(3)])).cuda()
    res = {}
    for fuse in (0, 1):
        with hh.Problem(2, n, ks, 0.0, ks, bc, hh.default_options(levels=3, fuse_sweeps=fuse)) as p:
            u, infos = p.solve(f, 1e-9)
            res[fuse] = (u.cpu(), [i.outer_its for i in infos])
    assert torch.equal(res[0][0], res[1][0]) and res[0][1] == res[1][1]


@pytest.mark.parametrize("prec", [hh.HH_C64, hh.HH_C128])
@pytest.mark.parametrize("n,levels,bc,nc", [(72, 4, (S, D, S, S), 8), (128, 3, (S, S, S, S), 8),
                                            (256, 3, (D, S, S, D), 8), (128, 3, (S, S, D, S), 7),
                                            (64, 2, (S, D, S, S), 1), (256, 3, (S, S, S, S), 2)])
def test_coarse_cluster_equals_separate_sweeps(libhh, prec, n, levels, bc, nc):
    """The coarsest level solved in one launch, by the thread-block cluster (sweeps in groups
    of up to four with recomputed halo rows: one-row slabs, groups of three and partial groups
    included) or by bands of rows with recomputed halos, equals
    the same sweeps run as separate kernels, bit for bit."""
    g = O.Grid(2, n, bc)
    r = torch.from_numpy(inputs.random_complex(g.N, 1500 + n) * g.free()).cuda()
    out = {}
    for name, cc, kern in (("separate", 0, 0), ("cluster", 100000, 1), ("bands", 100000, 2)):
        opts = hh.default_options(levels=levels, precision=prec, coarse_cluster_nodes=cc, nu_coarse=nc,
                                  coarse_kernel=kern)
        with hh.Problem(2, n, 12.0, 0.0, 12.0, bc, opts) as p:
            z = p.precondition(r)
            u, info = p.solve(r, 1e-9)
            out[name] = (z.cpu(), u.cpu(), info.outer_its)
    for name in ("cluster", "bands"):
        assert torch.equal(out["separate"][0], out[name][0]), name
        assert torch.equal(out["separate"][1], out[name][1]) and out["separate"][2] == out[name][2], name


@pytest.mark.parametrize("nb", [1, 3])
def test_coarse_bands_batch(libhh, nb):
    """Bands of rows and the cluster give the same bits, for a batch too."""
    n, bc = 128, (S, D, S, S)
    g = O.Grid(2, n, bc)
    ks = np.array([9.0, 14.0, 20.0])[:nb]
    r = torch.from_numpy(np.concatenate([inputs.random_complex(g.N, 1600 + b) * g.free() for b in range(nb)])).cuda()
    zs = []
    for kern in (1, 2):
        with hh.Problem(2, n, ks if nb > 1 else float(ks[0]), 0.0, ks if nb > 1 else float(ks[0]), bc,
                        hh.default_options(levels=3, coarse_kernel=kern)) as p:
            zs.append(p.precondition(r).cpu())
    assert torch.equal(zs[0], zs[1])
