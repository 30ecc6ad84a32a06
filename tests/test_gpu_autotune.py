"""Tile-shape autotuner: every tile shape computes each node the same way, so a tuned problem
must give bit-for-bit the result of an untuned one; the tuner must report the shapes it chose
and reuse them for a second problem of the same shape."""
import numpy as np
import pytest
import torch

from oracle import hh_oracle as O
from paper_2506_18694_gb300 import hh, inputs

pytestmark = pytest.mark.gpu

S, D = O.SOMMERFELD, O.DIRICHLET
MIX = [(10.0, 0.0, 10.0), (20.0, 0.0, 20.0), (20.0, 0.5, 2.0), (30.0, 0.0, 30.0)]


def _make(dim, n, bc, batch, **opt):
    if batch:
        ks, ds, dhs = (np.array(c) for c in zip(*MIX))
        return hh.Problem(dim, n, ks, ds, dhs, bc, hh.default_options(**opt))
    return hh.Problem(dim, n, 20.0, 0.0, 20.0, bc, hh.default_options(**opt))


@pytest.mark.parametrize("dim,n,bc,batch,prec", [
    (2, 128, (S, S, S, S), False, hh.HH_C64),
    (2, 128, (D, S, S, S), False, hh.HH_C128),
    (2, 64, (S, S, S, S), True, hh.HH_C64),
    (3, 16, (S, S, S, S, D, S), True, hh.HH_C64),
    (3, 24, (S, S, S, S, S, S), False, hh.HH_C64),
])
def test_tuned_solve_equals_untuned(libhh, dim, n, bc, batch, prec):
    g = O.Grid(dim, n, bc)
    nb = len(MIX) if batch else 1
    f = np.concatenate([inputs.random_complex(g.N, 1100 + b) * g.free() for b in range(nb)])
    opt = dict(levels=3, precision=prec)
    with _make(dim, n, bc, batch, **opt) as p0:
        u0, _ = p0.solve(torch.from_numpy(f).cuda(), 1e-9)
    with _make(dim, n, bc, batch, **opt) as p1:
        p1.solve(torch.from_numpy(f).cuda(), 1e-9)  # graph captured before tuning
        shapes = p1.autotune()
        u1, info = p1.solve(torch.from_numpy(f).cuda(), 1e-9)
    assert shapes, "nothing was tuned"
    for (l, mode), (rows, form) in shapes.items():
        if mode == "coarse":
            assert rows in (1, 2, 4, 8, 16) and form == 0 and l == 2
            continue
        if mode.endswith("_rr"):
            assert rows in (1, 2) and form == 1
            continue
        assert rows in (2, 4, 8) and form in (0, 1, 2)
        assert mode != "resid_restrict" or dim == 2
    assert torch.equal(u0, u1)
    # the same shape again: choices come from the process-wide record
    with _make(dim, n, bc, batch, autotune=1, **opt) as p2:
        assert p2.autotune() == shapes
        u2, _ = p2.solve(torch.from_numpy(f).cuda(), 1e-9)
    assert torch.equal(u0, u2)
