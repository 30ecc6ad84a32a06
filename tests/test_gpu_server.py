"""Continuous-batching server: requests of different grids, wavenumbers and boundary tags
submitted at once run concurrently under a device budget that forces queueing, pooling and
eviction; every result must equal, bit for bit, the lone solve of the same problem (the
kernels compute each node the same way whatever runs beside them), and the server's
accounting must respect its budget."""
import numpy as np
import pytest
import torch  # noqa: F401  (initialises the CUDA context the library uses)

from oracle import hh_oracle as O
from nodewise import rel
from paper_2506_18694_gb300 import hh, inputs

pytestmark = pytest.mark.gpu

S, D = O.SOMMERFELD, O.DIRICHLET

# dim, n, k, delta, delta_hat, bc
MIX = [
    (2, 64, 20.0, 0.0, 20.0, (S, S, S, S)),
    (2, 32, 10.0, 0.0, 2.0, (D, S, S, S)),
    (3, 16, 8.0, 0.0, 8.0, (S, S, S, S, D, S)),
    (2, 64, 30.0, 0.5, 30.0, (S, S, S, S)),      # same grid as the first: pooled problem reused
    (2, 128, 40.0, 0.0, 40.0, (S, S, D, S)),
    (3, 24, 12.0, 0.0, 12.0, (S, S, S, S, S, S)),
    (2, 32, 12.0, 0.0, 12.0, (D, S, S, S)),
    (2, 64, 25.0, 0.0, 25.0, (S, S, S, S)),
]


def _source(dim, n, seed):
    return inputs.gaussian_source(dim, n, tuple(np.random.default_rng(seed).uniform(0.2, 0.8, dim)), 0.05,
                                  complex(1.0, 0.5))


def _rhs(dim, n, bc, seed):
    return O.load_vector_nodal(O.Grid(dim, n, bc), _source(dim, n, seed))


NODAL = {2, 5}  # these requests pass the nodal source f; the server forms b = M f


@pytest.mark.timeout(600)
def test_server_mix_equals_alone(libhh):
    opts = hh.default_options(levels=3)
    fps = [hh.footprint_bytes(d, n, opts) for d, n, *_ in MIX]
    budget = sorted(fps)[-1] + sorted(fps)[-2]  # the two largest fit together, not everything
    rhs = [(_source(d, n, 900 + i) if i in NODAL else _rhs(d, n, bc, 900 + i))
           for i, (d, n, k, de, dh, bc) in enumerate(MIX)]
    with hh.Server(slots=3, budget_bytes=budget, options=opts) as srv:
        tickets = [srv.submit(d, n, k, de, dh, bc, rhs[i], 1e-9, nodal=i in NODAL)
                   for i, (d, n, k, de, dh, bc) in enumerate(MIX)]
        results = [srv.wait(t) for t in tickets]
        st = srv.stats()
    assert st["completed"] == len(MIX) and st["failed"] == 0
    assert st["peak_bytes"] <= budget
    assert st["max_concurrent"] >= 2
    assert st["problems_created"] + st["problems_reused"] == len(MIX)
    for i, (d, n, k, de, dh, bc) in enumerate(MIX):
        u, info, lat, qs = results[i]
        assert info.rel_residual <= 1e-9 and lat >= qs >= 0.0
        with hh.Problem(d, n, k, de, dh, bc, opts) as p:
            ua, ia = p.solve_host(rhs[i], 1e-9, nodal=i in NODAL)
        assert np.array_equal(u, ua), i
        assert info.outer_its == ia.outer_its and info.rel_residual == ia.rel_residual


@pytest.mark.timeout(300)
def test_server_retargets_pooled_problems(libhh):
    """One slot, same grid, new wavenumbers and shifts: the first request builds the problem,
    the others reuse it after hh_set_params; each result equals a fresh problem's."""
    opts = hh.default_options(levels=3)
    bc = (S, D, S, S)
    reqs = [(20.0, 0.0, 20.0), (12.0, 0.3, 2.0), (30.0, 0.0, 30.0)]
    rhs = [_rhs(2, 64, bc, 950 + i) for i in range(len(reqs))]
    with hh.Server(slots=1, budget_bytes=1 << 30, options=opts) as srv:
        res = [srv.wait(srv.submit(2, 64, k, de, dh, bc, rhs[i], 1e-9)) for i, (k, de, dh) in enumerate(reqs)]
        st = srv.stats()
    assert st["problems_created"] == 1 and st["problems_reused"] == 2 and st["max_concurrent"] == 1
    for i, (k, de, dh) in enumerate(reqs):
        with hh.Problem(2, 64, k, de, dh, bc, opts) as p:
            ua, ia = p.solve_host(rhs[i], 1e-9)
        assert np.array_equal(res[i][0], ua), i
        assert res[i][1].outer_its == ia.outer_its


@pytest.mark.timeout(300)
def test_server_rejects_what_never_fits(libhh):
    opts = hh.default_options(levels=3)
    small = hh.footprint_bytes(2, 32, opts)
    with hh.Server(slots=1, budget_bytes=small, options=opts) as srv:
        with pytest.raises(hh.HHError):
            srv.submit(2, 64, 10.0, 0.0, 10.0, (S, S, S, S), np.zeros(65 * 65, complex))
        t = srv.submit(2, 32, 10.0, 0.0, 10.0, (S, S, S, S), _rhs(2, 32, (S, S, S, S), 5))
        u, info, _, _ = srv.wait(t)
        assert info.rel_residual <= 1e-8
        with pytest.raises(hh.HHError):
            srv.wait(t)  # a ticket is waited for once


def _paper_multigrid(**kw):
    """The paper's multigrid (Sec. 5.3): W-cycles with GMRES(5) and a Jacobi preconditioner on
    every level, one cycle per HSS step (used at delta_hat = 2)."""
    return hh.default_options(cycle_gamma=2, nu_pre=5, nu_post=5, nu_coarse=5, smoother=hh.HH_SMOOTH_GMRES, **kw)


@pytest.mark.timeout(600)
def test_server_results_match_the_oracle(libhh):
    """Every served result against the FP64 oracle: its relative residual recomputed with the
    oracle's CSR matrix, and its solution error against sparse LU of the oracle's matrix."""
    opts = hh.default_options(levels=3)
    rhs = [_rhs(d, n, bc, 700 + i) for i, (d, n, k, de, dh, bc) in enumerate(MIX)]
    with hh.Server(slots=3, budget_bytes=4 << 30, options=opts) as srv:
        tickets = [srv.submit(d, n, k, de, dh, bc, rhs[i], 1e-9) for i, (d, n, k, de, dh, bc) in enumerate(MIX)]
        results = [srv.wait(t) for t in tickets]
    for i, (d, n, k, de, dh, bc) in enumerate(MIX):
        u, info, _, _ = results[i]
        prob = O.Problem(O.Grid(d, n, bc), k, de, dh, O.Options(levels=3))
        res = np.linalg.norm(rhs[i] - prob.B @ u) / np.linalg.norm(rhs[i])
        assert info.rel_residual <= 1e-9 and res <= 1.01e-9, i
        ex = prob.lu("B")(rhs[i])
        assert rel(u, ex) <= 1e-6, i


@pytest.mark.timeout(600)
def test_server_fallback_converges_what_the_first_settings_do_not(libhh):
    """A request whose first solve cannot converge (max_outer too small for V-cycles at
    delta_hat = k) is solved again with the fallback (the paper's multigrid at delta_hat = 2):
    it converges, reports the fallback, and equals both the lone fallback solve bit for bit
    and the oracle's LU solution; a request that converges at once does not fall back."""
    d, n, k, bc = 2, 64, 24.0, (S, S, S, S)
    first = hh.default_options(levels=3, max_outer=4, restart=4)
    fb = _paper_multigrid(levels=3, max_outer=300)
    hard = _rhs(d, n, bc, 801)
    with hh.Server(slots=2, budget_bytes=1 << 30, options=first) as srv:
        srv.set_fallback(fb, 2.0)
        u, info, _, _ = srv.wait(srv.submit(d, n, k, 0.0, k, bc, hard, 1e-9))
        zero_u, zero_info, _, _ = srv.wait(srv.submit(d, n, k, 0.0, k, bc, np.zeros_like(hard), 1e-9))
    assert info.fallback == 1 and info.rel_residual <= 1e-9 and info.outer_its > 4
    assert zero_info.fallback == 0 and np.all(zero_u == 0)
    with hh.Problem(d, n, k, 0.0, 2.0, bc, fb) as p:
        ua, ia = p.solve_host(hard, 1e-9)
    assert np.array_equal(u, ua) and info.outer_its == ia.outer_its + 4
    prob = O.Problem(O.Grid(d, n, bc), k, 0.0, 2.0, O.Options(levels=3))
    assert rel(u, prob.lu("B")(hard)) <= 1e-6


@pytest.mark.timeout(600)
def test_stall_detection_stops_early(libhh):
    """stall_cycles: FGMRES gives up once restart cycles stop halving the true residual."""
    d, n, k, bc = 2, 64, 24.0, (S, S, S, S)
    b = _rhs(d, n, bc, 802)
    # a tolerance below what FP64 arithmetic reaches: the residual levels off and stops halving
    with hh.Problem(d, n, k, 0.0, k, bc, hh.default_options(levels=3, max_outer=3000, stall_cycles=3)) as p:
        _, info = p.solve_host(b, 1e-18)
    assert info.rel_residual > 1e-18 and info.outer_its < 3000


@pytest.mark.timeout(600)
def test_server_pack_mode_equals_alone(libhh):
    """With a pack, the server's 2D requests of at most 25 HSS steps run as members of one pack
    (shared launches, slots refilled as members finish), the longer 2D ones and the 3D ones on
    the worker slots; every result equals its lone solve bit for bit, and the budget holds."""
    opts = hh.default_options(levels=3)
    fps = [hh.footprint_bytes(d, n, opts) for d, n, *_ in MIX]
    budget = 3 * sorted(fps)[-1]
    rhs = [(_source(d, n, 1900 + i) if i in NODAL else _rhs(d, n, bc, 1900 + i))
           for i, (d, n, k, de, dh, bc) in enumerate(MIX)]
    with hh.Server(slots=2, budget_bytes=budget, options=opts) as srv:
        srv.set_pack(3, 25)
        tickets = [srv.submit(d, n, k, de, dh, bc, rhs[i], 1e-9, nodal=i in NODAL)
                   for i, (d, n, k, de, dh, bc) in enumerate(MIX)]
        results = [srv.wait(t) for t in tickets]
        st = srv.stats()
    assert st["completed"] == len(MIX) and st["failed"] == 0 and st["peak_bytes"] <= budget
    for i, (d, n, k, de, dh, bc) in enumerate(MIX):
        u, info, lat, qs = results[i]
        assert info.rel_residual <= 1e-9 and lat >= qs >= 0.0
        with hh.Problem(d, n, k, de, dh, bc, opts) as p:
            ua, ia = p.solve_host(rhs[i], 1e-9, nodal=i in NODAL)
        assert np.array_equal(u, ua), i
        assert info.outer_its == ia.outer_its, i
