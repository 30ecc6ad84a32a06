"""Packs: FGMRES solves of problems on DIFFERENT grids whose preconditioner applications share
launches (one launch per V-cycle pass over the tiles of every member), through the C ABI.

Every member's iteration is the sequence of operations of its own solve, so each result must
equal that problem's lone hh_solve bit for bit (same iterate, iteration count and residual);
the oracle checks the results against sparse LU of its assembled matrix.  Members that finish
leave and their slots are refilled while the others keep running (continuous batching).
"""
import numpy as np
import pytest
import torch

from nodewise import rel
from oracle import hh_oracle as O
from paper_2506_18694_gb300 import hh, inputs

pytestmark = pytest.mark.gpu

S, D = O.SOMMERFELD, O.DIRICHLET

# n, k, delta, delta_hat, bc: four grids, four wavenumbers, both boundary layouts
MEMBERS = [
    (64, 12.0, 0.0, 12.0, (S, S, S, S)),
    (96, 20.0, 0.2, 20.0, (D, S, S, D)),
    (128, 9.0, 0.0, 2.0, (S, S, D, S)),
    (40, 6.0, 0.0, 6.0, (S, D, S, S)),
    (256, 30.0, 0.0, 30.0, (S, S, S, S)),
    (72, 15.0, 0.0, 15.0, (S, S, S, S)),
]
TOL = 1e-9


def _rhs(n, bc, seed):
    g = O.Grid(2, n, bc)
    f = inputs.gaussian_source(2, n, tuple(np.random.default_rng(seed).uniform(0.2, 0.8, 2)), 0.05, complex(1.0, 0.3))
    return O.load_vector_nodal(g, f), f


def _lone(n, k, de, dh, bc, b):
    with hh.Problem(2, n, k, de, dh, bc, hh.default_options()) as p:
        u, info = p.solve(torch.from_numpy(b).cuda(), TOL)
        return u.cpu().numpy(), info


def test_pack_equals_lone_solves_and_oracle(libhh):
    rhs = [_rhs(n, bc, 60 + i)[0] for i, (n, k, de, dh, bc) in enumerate(MEMBERS)]
    probs = [hh.Problem(2, n, k, de, dh, bc, hh.default_options()) for n, k, de, dh, bc in MEMBERS]
    got = {}
    try:
        with hh.Pack(capacity=len(MEMBERS)) as pk:
            slots = {pk.add(p, torch.from_numpy(b).cuda(), TOL): i for i, (p, b) in enumerate(zip(probs, rhs))}
            while pk.members():
                for s in pk.run():
                    u, info = pk.take(s)
                    got[slots[s]] = (u.cpu().numpy(), info)
    finally:
        for p in probs:
            p.close()
    assert sorted(got) == list(range(len(MEMBERS)))
    for i, (n, k, de, dh, bc) in enumerate(MEMBERS):
        u, info = got[i]
        ul, il = _lone(n, k, de, dh, bc, rhs[i])
        assert np.array_equal(u, ul), i
        assert info.outer_its == il.outer_its and info.rel_residual == il.rel_residual <= TOL, i
        assert info.vcycles == il.vcycles
        if n <= 128:
            prob = O.Problem(O.Grid(2, n, bc), k, de, dh, O.Options())
            assert rel(u, prob.lu("B")(rhs[i])) <= 1e-6, i


def test_pack_refills_finished_slots(libhh):
    """Capacity 2, six requests: each finished member's slot is refilled at once; every result
    still equals its lone solve, and the pack never holds more than two members."""
    rhs = [_rhs(n, bc, 80 + i) for i, (n, k, de, dh, bc) in enumerate(MEMBERS)]
    queue = list(range(len(MEMBERS)))
    probs, got, slot_of = {}, {}, {}
    with hh.Pack(capacity=2) as pk:
        def admit():
            while queue and pk.members() < 2:
                i = queue.pop(0)
                n, k, de, dh, bc = MEMBERS[i]
                probs[i] = hh.Problem(2, n, k, de, dh, bc, hh.default_options())
                slot_of[pk.add(probs[i], rhs[i][1], TOL, nodal=True)] = i  # host nodal source
        admit()
        while pk.members():
            for s in pk.run():
                i = slot_of.pop(s)
                got[i] = pk.take(s)
                probs.pop(i).close()
            assert pk.members() <= 2
            admit()
    for i, (n, k, de, dh, bc) in enumerate(MEMBERS):
        u, info = got[i]
        with hh.Problem(2, n, k, de, dh, bc, hh.default_options()) as p:
            ul, il = p.solve_host(rhs[i][1], TOL, nodal=True)
        assert np.array_equal(u, ul), i
        assert info.outer_its == il.outer_its, i


def test_pack_rejects_what_it_cannot_run(libhh):
    with hh.Pack(capacity=1) as pk, \
            hh.Problem(3, 16, 5.0, 0.0, 5.0, (S,) * 6, hh.default_options(levels=3)) as p3, \
            hh.Problem(2, 32, 5.0, 0.0, 5.0, (S,) * 4, hh.default_options(cycle_gamma=2)) as pw, \
            hh.Problem(2, 32, 5.0, 0.0, 5.0, (S,) * 4, hh.default_options()) as a, \
            hh.Problem(2, 32, 5.0, 0.0, 5.0, (S,) * 4, hh.default_options()) as b:
        z = torch.zeros(33 * 33, dtype=torch.complex128, device="cuda")
        for bad in (p3, pw):
            with pytest.raises(hh.HHError):
                pk.add(bad, torch.zeros(bad.system_size(), dtype=torch.complex128, device="cuda"))
        pk.add(a, z)
        with pytest.raises(hh.HHError):
            pk.add(b, z)  # full
        s = pk.run()
        u, info = pk.take(s[0])
        assert info.outer_its == 0 and torch.count_nonzero(u) == 0  # zero right side: u = 0
