"""GPU parity: every kernel and the whole solver, through the C ABI, against the FP64 oracle.

Tolerances, on the larger of the norm-wise error ||gpu - oracle|| / ||oracle|| and the per-node
error max|gpu - oracle| / max|oracle| (nodewise.rel; Dirichlet nodes must hold exact zeros):
  complex128 kernels  1e-12   (the same sums in a different order: rounding only)
  complex64 kernels   2e-6    (a 9/27-term stencil in FP32: a few ulps of 6e-8 each)
  complex64 V-cycle   2e-5    (about 20 FP32 stencil passes)
  solves              relative residual <= tol (FP64, recomputed by the oracle's CSR matrix)
                      and solution error <= 1e-6 against sparse LU
"""
import numpy as np
import pytest
import torch

from oracle import hh_oracle as O
from nodewise import rel
from paper_2506_18694_gb300 import hh, inputs

pytestmark = pytest.mark.gpu

S, D = O.SOMMERFELD, O.DIRICHLET
TOL = {hh.HH_C128: 1e-12, hh.HH_C64: 2e-6}
DT = {hh.HH_C128: torch.complex128, hh.HH_C64: torch.complex64}

CASES = [
    # dim, n, levels, bc  (n=72 -> 73 nodes/axis: ragged against 32x8 thread tiles)
    (2, 8, 3, (S, S, S, S)),
    (2, 72, 4, (S, S, S, S)),
    (2, 72, 3, (D, S, S, D)),
    (2, 16, 3, (S, D, D, S)),
    (3, 8, 3, (S, S, S, S, D, S)),
    (3, 12, 3, (D, D, S, S, S, D)),
    (3, 16, 3, (S, S, S, S, S, S)),
    (3, 64, 3, (S, S, D, S, D, S)),  # 65^3: interior 3D tiles take the check-free path
]
K_, DELTA, DHAT = 7.0, 0.3, 2.5




def to_dev(v, prec):
    return torch.from_numpy(np.ascontiguousarray(v)).to(DT[prec]).cuda()


def to_np(t):
    return t.cpu().numpy().astype(np.complex128)


@pytest.fixture(scope="module", params=CASES, ids=lambda c: f"d{c[0]}n{c[1]}L{c[2]}bc{''.join(map(str, c[3]))}")
def case(request, libhh):
    dim, n, L, bc = request.param
    g = O.Grid(dim, n, bc)
    prob = O.Problem(g, K_, DELTA, DHAT, O.Options(levels=L, omega=0.6, nu_pre=2, nu_post=2, nu_coarse=8))
    opts = hh.default_options(levels=L, omega=0.6, nu_pre=2, nu_post=2, nu_coarse=8)
    p = hh.Problem(dim, n, K_, DELTA, DHAT, bc, opts)
    yield g, prob, p
    p.close()


def rand(g, seed):
    return inputs.random_complex(g.N, seed) * g.free()


def oracle_op(prob, l, op):
    mats = prob.mats[l]
    k, dh, delta = prob.k, prob.delta_hat, prob.delta
    table = {
        "K": (1, 0, 0), "M": (0, 1, 0), "MGAMMA": (0, 0, 1),
        "AL": O.coeff_AL(k, dh), "AR": O.coeff_AR(k, dh), "B": O.coeff_B(k, delta),
        "BHAT": O.coeff_B(k, dh),
    }
    return O.combine(mats, table[op])


@pytest.mark.parametrize("prec", [hh.HH_C128, hh.HH_C64])
@pytest.mark.parametrize("op", ["K", "M", "MGAMMA", "AL", "AR", "B", "BHAT"])
def test_apply(case, op, prec):
    g, prob, p = case
    for l in range(len(prob.grids)):
        gl = prob.grids[l]
        x = inputs.random_complex(gl.N, 11 + l)  # Dirichlet entries nonzero on purpose: ignored
        y = to_np(p.apply(l, op, to_dev(x, prec)))
        ref = oracle_op(prob, l, op) @ (x * gl.free())
        assert rel(y, ref) <= TOL[prec], (l, rel(y, ref))
        assert np.all(y[~gl.free()] == 0)


@pytest.mark.parametrize("prec", [hh.HH_C128, hh.HH_C64])
def test_jacobi(case, prec):
    g, prob, p = case
    for l in range(len(prob.grids)):
        gl = prob.grids[l]
        b = rand(gl, 20 + l)
        x = rand(gl, 30 + l)
        y = to_np(p.jacobi(l, to_dev(b, prec), to_dev(x, prec)))
        assert rel(y, prob.jacobi(l, b, x)) <= TOL[prec]
        y0 = to_np(p.jacobi(l, to_dev(b, prec), None))
        assert rel(y0, prob.jacobi(l, b, np.zeros_like(b))) <= TOL[prec]


@pytest.mark.parametrize("prec", [hh.HH_C128, hh.HH_C64])
def test_residual_restrict_and_prolong(case, prec):
    g, prob, p = case
    for l in range(len(prob.grids) - 1):
        gl, gc = prob.grids[l], prob.grids[l + 1]
        b, x = rand(gl, 40 + l), rand(gl, 50 + l)
        rc = to_np(p.residual_restrict(l, to_dev(b, prec), to_dev(x, prec)))
        ref = prob.P[l].T @ (b - prob.AL[l] @ x)
        assert rel(rc, ref) <= TOL[prec] * 10
        ec = rand(gc, 60 + l)
        xd = to_dev(x, prec)
        out = to_np(p.prolong_correct(l, to_dev(ec, prec), xd))
        assert rel(out, x + prob.P[l] @ ec) <= TOL[prec]


@pytest.mark.parametrize("prec", [hh.HH_C128, hh.HH_C64])
def test_vcycle(case, prec):
    g, prob, p = case
    b = rand(g, 70)
    x = to_np(p.vcycle(to_dev(b, prec)))
    assert rel(x, prob.vcycle(0, b)) <= (1e-12 if prec == hh.HH_C128 else 2e-5)


NU = [(2, 2, 8), (1, 1, 3), (3, 2, 0), (0, 1, 2), (2, 0, 5), (4, 3, 1)]


@pytest.mark.parametrize("prec", [hh.HH_C128, hh.HH_C64])
@pytest.mark.parametrize("nu", NU, ids=lambda v: "nu%d%d%d" % v)
@pytest.mark.parametrize("dim,n,L,bc", [(2, 40, 4, (S, D, S, S)), (3, 8, 3, (S, S, D, S, S, S))])
def test_vcycle_sweep_counts(libhh, prec, nu, dim, n, L, bc):
    """Every pre/post/coarse sweep count takes a different fused-kernel path."""
    g = O.Grid(dim, n, bc)
    o = dict(levels=L, nu_pre=nu[0], nu_post=nu[1], nu_coarse=nu[2], omega=0.7)
    prob = O.Problem(g, 5.0, 0.0, 3.0, O.Options(**o))
    with hh.Problem(dim, n, 5.0, 0.0, 3.0, bc, hh.default_options(**o)) as p:
        b = rand(g, 71)
        x = to_np(p.vcycle(to_dev(b, prec)))
    assert rel(x, prob.vcycle(0, b)) <= (1e-12 if prec == hh.HH_C128 else 2e-5)


@pytest.mark.parametrize("prec", [hh.HH_C128, hh.HH_C64])
@pytest.mark.parametrize("pdl,cluster", [(0, 0), (1, 0), (0, 20000), (1, 100000)])
@pytest.mark.parametrize("dim,n,L,bc", [(2, 64, 4, (D, S, S, S)), (3, 16, 4, (S, S, S, S, D, S))])
def test_vcycle_launch_modes(libhh, prec, pdl, cluster, dim, n, L, bc):
    """Same V-cycle with and without programmatic launch and the cluster-resident bottom."""
    g = O.Grid(dim, n, bc)
    prob = O.Problem(g, 8.0, 0.0, 8.0, O.Options(levels=L))
    opts = hh.default_options(levels=L, use_pdl=pdl, coarse_cluster_nodes=cluster)
    with hh.Problem(dim, n, 8.0, 0.0, 8.0, bc, opts) as p:
        b = rand(g, 72)
        x = to_np(p.vcycle(to_dev(b, prec)))
        x2 = to_np(p.vcycle(to_dev(b, prec)))
    assert rel(x, prob.vcycle(0, b)) <= (1e-12 if prec == hh.HH_C128 else 2e-5)
    assert np.array_equal(x, x2)  # deterministic


@pytest.mark.parametrize("prec", [hh.HH_C128, hh.HH_C64])
@pytest.mark.parametrize("rows", [2, 4, 8])
@pytest.mark.parametrize("dim,n,bc", [(2, 72, (S, D, S, S)), (3, 24, (S, S, D, S, S, S))])
def test_tile_rows(libhh, prec, rows, dim, n, bc):
    """Every tile height gives the same apply, sweep and residual-restriction."""
    g = O.Grid(dim, n, bc)
    prob = O.Problem(g, 6.0, 0.0, 3.0, O.Options(levels=2))
    with hh.Problem(dim, n, 6.0, 0.0, 3.0, bc, hh.default_options(levels=2, tile_rows=rows)) as p:
        x, b = rand(g, 110), rand(g, 111)
        assert rel(to_np(p.apply(0, "AL", to_dev(x, prec))), prob.AL[0] @ x) <= TOL[prec]
        assert rel(to_np(p.jacobi(0, to_dev(b, prec), to_dev(x, prec))), prob.jacobi(0, b, x)) <= TOL[prec]
        rc = to_np(p.residual_restrict(0, to_dev(b, prec), to_dev(x, prec)))
        assert rel(rc, prob.P[0].T @ (b - prob.AL[0] @ x)) <= TOL[prec] * 10


@pytest.mark.parametrize("prec", [hh.HH_C128, hh.HH_C64])
@pytest.mark.parametrize("nu", [(2, 2, 8), (0, 1, 2), (1, 0, 4)], ids=lambda v: "nu%d%d%d" % v)
@pytest.mark.parametrize("cycles", [1, 2])
def test_precondition_paths(libhh, prec, nu, cycles):
    """HSS loop with and without the fused first sweep, one or two V-cycles per HSS step."""
    g = O.Grid(2, 32, (S, S, S, D))
    o = dict(levels=3, nu_pre=nu[0], nu_post=nu[1], nu_coarse=nu[2], cycles_per_hss=cycles)
    prob = O.Problem(g, 4.5, 0.0, 2.0, O.Options(**o))
    with hh.Problem(2, 32, 4.5, 0.0, 2.0, g.bc, hh.default_options(precision=prec, **o)) as p:
        r = rand(g, 101)
        z = to_np(p.precondition(to_dev(r, hh.HH_C128)))
    assert rel(z, prob.prec(r)) <= (1e-11 if prec == hh.HH_C128 else 5e-5)


@pytest.mark.parametrize("prec", [hh.HH_C128, hh.HH_C64])
def test_hss_rhs(case, prec):
    g, prob, p = case
    u, r = rand(g, 80), rand(g, 81)
    out = to_np(p.hss_rhs(to_dev(u, prec), to_dev(r, prec)))
    assert rel(out, prob.hss_rhs(u, r)) <= TOL[prec]
    out0 = to_np(p.hss_rhs(None, to_dev(r, prec)))
    assert rel(out0, prob.hss_rhs(np.zeros_like(r), r)) <= TOL[prec]


def test_load_vector_and_dot(case):
    g, prob, p = case
    f = inputs.random_complex(g.N, 90)
    b = to_np(p.load_vector(to_dev(f, hh.HH_C128)))
    assert rel(b, prob.mats[0][1] @ (f * g.free())) <= 1e-13
    x, y = inputs.random_complex(g.N, 91), inputs.random_complex(g.N, 92)
    d = p.dot(to_dev(x, hh.HH_C128), to_dev(y, hh.HH_C128))
    ref = np.vdot(x, y)
    assert abs(d - ref) <= 1e-13 * np.linalg.norm(x) * np.linalg.norm(y)


@pytest.mark.parametrize("prec,graphs", [(hh.HH_C128, 0), (hh.HH_C128, 1), (hh.HH_C64, 1)])
def test_precondition(prec, graphs, libhh):
    g = O.Grid(2, 32, (S, S, D, S))
    prob = O.Problem(g, 6.0, 0.0, 2.0, O.Options(levels=3))
    opts = hh.default_options(levels=3, precision=prec, use_graphs=graphs)
    with hh.Problem(2, 32, 6.0, 0.0, 2.0, g.bc, opts) as p:
        r = rand(g, 100)
        z1 = to_np(p.precondition(to_dev(r, hh.HH_C128)))
        z2 = to_np(p.precondition(to_dev(r, hh.HH_C128)))  # replay
        ref = prob.prec(r)
        tol = 1e-11 if prec == hh.HH_C128 else 5e-5
        assert rel(z1, ref) <= tol and rel(z2, ref) <= tol


SOLVES = [
    # dim, n, k, delta, delta_hat, bc, levels
    (2, 32, 10.0, 0.0, 10.0, (S, S, S, S), 4),   # the 32^2, k=10 workload (delta_hat = k)
    (2, 32, 10.0, 0.0, 2.0, (S, S, S, S), 4),    # the paper's delta_hat = 2
    (2, 64, 12.0, 0.5, 2.0, (D, S, S, S), 3),
    (3, 16, 6.0, 0.0, 2.0, (S, S, S, S, D, S), 3),
]


@pytest.mark.parametrize("prec", [hh.HH_C128, hh.HH_C64])
@pytest.mark.parametrize("dim,n,k,delta,dh,bc,L", SOLVES)
def test_solve_matches_lu(libhh, prec, dim, n, k, delta, dh, bc, L):
    g = O.Grid(dim, n, bc)
    prob = O.Problem(g, k, delta, dh, O.Options(levels=L))
    c = (0.5,) * dim
    f = inputs.gaussian_source(dim, n, c, 0.05)
    b = O.load_vector_nodal(g, f)
    ex = prob.lu("B")(b)
    opts = hh.default_options(levels=L, precision=prec)
    with hh.Problem(dim, n, k, delta, dh, bc, opts) as p:
        bd = p.load_vector(to_dev(f, hh.HH_C128))
        assert rel(to_np(bd), b) <= 1e-13
        u, info = p.solve(bd, tol=1e-8)
        u = to_np(u)
    res = np.linalg.norm(b - prob.B @ u) / np.linalg.norm(b)
    assert info.rel_residual <= 1e-8 and res <= 1.01e-8
    assert abs(res - info.rel_residual) <= 1e-10
    assert rel(u, ex) <= 1e-6
    if (~g.free()).any():
        assert np.all(u[~g.free()] == 0)
    if prec == hh.HH_C128:
        # same algorithm in FP64: outer iteration counts agree within one
        _, its, _, _ = O.solve(prob, b, 1e-8)
        assert abs(info.outer_its - its) <= 1, (info.outer_its, its)
        assert info.hss_its == info.outer_its * O.n_hss(k)


def test_solve_host_buffers_match_device(libhh):
    w = inputs.workload("2d_n32_k10")
    f = inputs.gaussian_source(w.dim, w.n, w.centre, w.sigma)
    with hh.Problem(w.dim, w.n, w.k, w.delta, w.delta_hat, w.bc) as p:
        b = p.load_vector(to_dev(f, hh.HH_C128))
        u_dev, i1 = p.solve(b, 1e-8)
        u_host, i2 = p.solve_host(b.cpu().numpy(), 1e-8)
    assert i1.outer_its == i2.outer_its
    assert np.array_equal(to_np(u_dev), u_host)  # same kernels, same order: bitwise equal


def test_solve_zero_rhs_and_initial_guess(libhh):
    g = O.Grid(2, 16, (S,) * 4)
    with hh.Problem(2, 16, 5.0, 0.0, 2.0, g.bc, hh.default_options(levels=3)) as p:
        z = p.zeros()
        u, info = p.solve(z, 1e-8)
        assert info.rel_residual == 0.0 and torch.count_nonzero(u).item() == 0
        f = to_dev(inputs.gaussian_source(2, 16, (0.3, 0.6)), hh.HH_C128)
        b = p.load_vector(f)
        u1, i1 = p.solve(b, 1e-8)
        u2, i2 = p.solve(b, 1e-8, x0=u1)  # resume from the converged answer
        assert i2.outer_its == 0 and i2.rel_residual <= 1e-8


def test_allocation_limit_injects_oom(libhh):
    """A per-problem device cap fails creation with HH_ERR_OOM before any allocation (no
    device fault, nothing leaked), and lifting it lets the same problem be created and solved."""
    lib = hh.load_library()
    opts = hh.default_options(levels=3)
    need = hh.footprint_bytes(2, 16, opts)
    try:
        lib.hh_set_allocation_limit(need // 2)
        with pytest.raises(hh.HHError) as e:
            hh.Problem(2, 16, 5.0, 0.0, 2.0, (S,) * 4, opts)
        assert e.value.status == -2 and "limit" in str(e.value)
        lib.hh_set_allocation_limit(need)
        with hh.Problem(2, 16, 5.0, 0.0, 2.0, (S,) * 4, opts) as p:
            b = p.load_vector(to_dev(inputs.gaussian_source(2, 16, (0.5, 0.5)), hh.HH_C128))
            _, info = p.solve(b, 1e-8)
            assert info.rel_residual <= 1e-8 and info.device_bytes <= need
    finally:
        lib.hh_set_allocation_limit(0)


def test_nonfinite_rhs_reported(libhh):
    with hh.Problem(2, 16, 5.0, 0.0, 2.0, (S,) * 4, hh.default_options(levels=3)) as p:
        b = p.zeros()
        b[40] = complex(float("nan"), 0.0)
        with pytest.raises(hh.HHError) as e:
            p.solve(b, 1e-8)
        assert e.value.status == -4
        # the problem stays usable
        b2 = p.load_vector(to_dev(inputs.gaussian_source(2, 16, (0.5, 0.5)), hh.HH_C128))
        _, info = p.solve(b2, 1e-8)
        assert info.rel_residual <= 1e-8
