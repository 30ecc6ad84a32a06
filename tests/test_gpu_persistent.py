"""The persistent HSS loop (one cooperative kernel per preconditioner application, grid-wide
barriers between the passes of each V-cycle) against the one-kernel-per-pass path and the
oracle, through the C ABI.

Both paths compute every node with the same device arithmetic, so their results must agree
bit for bit; the oracle checks both against Def. 4.1.  A grid-barrier wait that is made to run
out (a spin limit of one poll) must return HH_ERR_TIMEOUT and leave the device usable.
"""
import numpy as np
import pytest
import torch

from nodewise import rel
from oracle import hh_oracle as O
from paper_2506_18694_gb300 import hh, inputs

pytestmark = pytest.mark.gpu

S, D = O.SOMMERFELD, O.DIRICHLET
DT = {hh.HH_C128: torch.complex128, hh.HH_C64: torch.complex64}


def _pair(dim, n, k, delta, dh, bc, **kw):
    on = hh.Problem(dim, n, k, delta, dh, bc, hh.default_options(persistent=2, **kw))
    off = hh.Problem(dim, n, k, delta, dh, bc, hh.default_options(persistent=0, **kw))
    return on, off


@pytest.mark.parametrize("prec", [hh.HH_C64, hh.HH_C128])
@pytest.mark.parametrize("n,L,bc,nu_c", [
    (8, 2, (S, S, S, S), 8),
    (72, 4, (S, S, S, S), 8),
    (72, 3, (D, S, S, D), 3),
    (48, 4, (S, D, D, S), 1),
    (64, 5, (D, D, S, S), 8),
])
def test_preconditioner_bitwise_and_oracle(libhh, prec, n, L, bc, nu_c):
    k, delta, dh = 7.0, 0.3, 2.5
    g = O.Grid(2, n, bc)
    prob = O.Problem(g, k, delta, dh, O.Options(levels=L, omega=0.6, nu_coarse=nu_c))
    r = inputs.random_complex(g.N, 31) * g.free()
    ref = prob.prec(r)
    on, off = _pair(2, n, k, delta, dh, bc, levels=L, precision=prec, nu_coarse=nu_c)
    try:
        rd = torch.from_numpy(r).cuda()
        z_on = on.precondition(rd)
        z_off = off.precondition(rd)
        z_on2 = on.precondition(rd)  # a second launch reuses the plan and the barrier words
        torch.cuda.synchronize()
    finally:
        on.close()
        off.close()
    assert torch.equal(z_on, z_off)
    assert torch.equal(z_on, z_on2)
    tol = 1e-11 if prec == hh.HH_C128 else 5e-5
    assert rel(z_on.cpu().numpy(), ref) <= tol


def test_batch_bitwise_uneven_hss_lengths(libhh):
    """Three problems with different k (hence HSS lengths 5, 9, 12) in one batch."""
    n, bc = 64, (S, S, S, S)
    ks = np.array([5.0, 9.0, 12.0])
    dh = np.array([2.0, 9.0, 3.0])
    N = (n + 1) ** 2
    r = torch.from_numpy(np.concatenate([inputs.random_complex(N, 40 + i) for i in range(3)])).cuda()
    on = hh.Problem(2, n, ks, 0.0, dh, bc, hh.default_options(persistent=2))
    off = hh.Problem(2, n, ks, 0.0, dh, bc, hh.default_options(persistent=0))
    try:
        z_on = on.precondition(r)
        z_off = off.precondition(r)
        torch.cuda.synchronize()
    finally:
        on.close()
        off.close()
    assert torch.equal(z_on, z_off)
    g = O.Grid(2, n, bc)
    for b in range(3):
        prob = O.Problem(g, float(ks[b]), 0.0, float(dh[b]), O.Options())
        ref = prob.prec(r[b * N:(b + 1) * N].cpu().numpy())
        assert rel(z_on[b * N:(b + 1) * N].cpu().numpy(), ref) <= 5e-5, b


def test_c2_solve_bitwise_and_fewer_launches(libhh):
    """The 2D 512^2, k = 80 workload: the same iterate, iteration count and residual with both
    forms; the persistent form launches one kernel per HSS loop instead of seven per V-cycle."""
    w = inputs.workload("2d_n512_k80")
    f = torch.from_numpy(inputs.gaussian_source(w.dim, w.n, w.centre, w.sigma)).cuda()
    on, off = _pair(w.dim, w.n, w.k, w.delta, w.delta_hat, w.bc)
    try:
        b = on.load_vector(f)
        u_on, i_on = on.solve(b, w.tol)
        u_off, i_off = off.solve(b, w.tol)
        torch.cuda.synchronize()
    finally:
        on.close()
        off.close()
    assert i_on.outer_its == i_off.outer_its and i_on.vcycles == i_off.vcycles
    assert i_on.rel_residual == i_off.rel_residual <= w.tol
    assert torch.equal(u_on, u_off)
    assert i_on.kernel_launches * 20 < i_off.kernel_launches


def test_barrier_timeout_returns_and_device_stays_usable(libhh):
    """A spin limit of one poll makes the grid-barrier waits run out on purpose: the kernel
    records HH_ERR_TIMEOUT and returns (no hang); the call reports it; the context and a fresh
    problem then work normally."""
    n, bc = 64, (S, S, S, S)
    N = (n + 1) ** 2
    r = torch.from_numpy(inputs.random_complex(N, 50)).cuda()
    p = hh.Problem(2, n, 9.0, 0.0, 9.0, bc, hh.default_options(persistent=2, sync_spin_limit=1))
    try:
        with pytest.raises(hh.HHError) as e:
            p.precondition(r)
        assert e.value.status == hh.HH_ERR_TIMEOUT
        with pytest.raises(hh.HHError) as e:
            p.solve(r, 1e-8)
        assert e.value.status == hh.HH_ERR_TIMEOUT
    finally:
        p.close()
    torch.cuda.synchronize()
    on, off = _pair(2, n, 9.0, 0.0, 9.0, bc)
    try:
        assert torch.equal(on.precondition(r), off.precondition(r))
    finally:
        on.close()
        off.close()
