"""p-multigrid preconditioner (Chebyshev-Jacobi smoothing, GLL-to-GLL
transfers, rediscretised levels on the eta-following geometry): the
preconditioned solves reach the same discrete solution as the oracle, in FP64
and inside the mixed-precision defect correction, with far fewer iterations
than Jacobi."""
import numpy as np
import pytest
import torch

from oracle import solve as osolve
from oracle import surface as osurf
from tests.pairs import Case, rel_l2
from tests.test_gpu_parity import SHAPES, ids

pytestmark = pytest.mark.gpu


def pmg(fnpf, rtol=1e-13, **kw):
    return fnpf.default_opts(precond=fnpf.FNPF_PMG, rtol=rtol, max_iter=5000, **kw)


@pytest.mark.parametrize("shape", SHAPES, ids=ids)
def test_pmg_solve_matches_oracle(fnpf, shape):
    c = Case(fnpf, *shape, opts=pmg(fnpf))
    phi_ref = osolve.laplace_solve(c.om, c.eta, c.h, c.phis)
    phi = torch.zeros(c.om.N, dtype=torch.float64, device=c.dev)
    info = c.gm.laplace_solve(c.t(c.eta), c.t(c.phis), phi)
    assert info["status"] == 0 and info["rel_res"] <= 1e-13
    assert rel_l2(phi.cpu().numpy(), phi_ref) < 1e-10


@pytest.mark.parametrize("shape", [SHAPES[0], SHAPES[2], SHAPES[3], SHAPES[5]], ids=ids)
def test_pmg_mixed_solve_matches_oracle(fnpf, shape):
    c = Case(fnpf, *shape, opts=pmg(fnpf, precision=fnpf.FNPF_MIXED, inner_rtol=1e-5))
    phi_ref = osolve.laplace_solve(c.om, c.eta, c.h, c.phis)
    phi = torch.zeros(c.om.N, dtype=torch.float64, device=c.dev)
    info = c.gm.laplace_solve(c.t(c.eta), c.t(c.phis), phi)
    assert info["status"] == 0 and info["rel_res"] <= 1e-13
    assert rel_l2(phi.cpu().numpy(), phi_ref) < 1e-10


def test_pmg_needs_far_fewer_iterations_than_jacobi(fnpf):
    shape = (3, 8, 8, 2, 6, True, True)
    cj = Case(fnpf, *shape, h0=0.3, opts=fnpf.default_opts(rtol=1e-10))
    cp = Case(fnpf, *shape, h0=0.3, opts=pmg(fnpf, rtol=1e-10))
    phi = torch.zeros(cj.om.N, dtype=torch.float64, device=cj.dev)
    ij = cj.gm.laplace_solve(cj.t(cj.eta), cj.t(cj.phis), phi)["iters"]
    phi.zero_()
    ip = cp.gm.laplace_solve(cp.t(cp.eta), cp.t(cp.phis), phi)["iters"]
    assert ip * 5 < ij, (ip, ij)


def test_pmg_rk4_matches_oracle(fnpf):
    c = Case(fnpf, 3, 5, 3, 2, 4, True, False, opts=pmg(fnpf))
    dt = 0.01
    eta_r, phi_r = c.eta.copy(), c.phis.copy()
    eta, phis = c.t(c.eta), c.t(c.phis)
    for _ in range(2):
        eta_r, phi_r = osurf.rk4_step(c.om, c.h, eta_r, phi_r, dt, 9.81)
        c.gm.rk4_step(eta, phis, 0.0, dt)
    torch.cuda.synchronize()
    assert rel_l2(eta.cpu().numpy(), eta_r) < 1e-10
    assert rel_l2(phis.cpu().numpy(), phi_r) < 1e-10


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_graph_replay_is_bitwise_identical_to_plain_launches(fnpf, precision):
    """CUDA-graph replay of the CG iterations runs the same kernels with the
    same arguments: results match plain launches bit for bit."""
    prec = fnpf.FNPF_MIXED if precision == "mixed" else fnpf.FNPF_FP64
    shape = (3, 6, 5, 2, 5, True, False)
    out = []
    for graphs in (0, 1):
        c = Case(fnpf, *shape, opts=pmg(fnpf, rtol=1e-12, precision=prec, use_graphs=graphs, check_every=4))
        c.gm.set_shapes(1, 1)   # the same kernels on both meshes (the autotuner could pick different ones)
        eta, phis = c.t(c.eta), c.t(c.phis)
        for _ in range(2):
            c.gm.rk4_step(eta, phis, 0.0, 0.01)
        torch.cuda.synchronize()
        out.append((eta.cpu().numpy(), phis.cpu().numpy()))
    assert np.array_equal(out[0][0], out[1][0]) and np.array_equal(out[0][1], out[1][1])


@pytest.mark.parametrize("precond", ["jacobi", "pmg"])
def test_stored_metric_matches_on_the_fly_metric(fnpf, precond):
    """FP64 solves reading the metric stored once per solve give the solution
    of the solves that rebuild it per application (and of the oracle)."""
    pre = fnpf.FNPF_PMG if precond == "pmg" else fnpf.FNPF_JACOBI
    shape = (3, 5, 4, 2, 5, True, False)
    sol = []
    for store in (0, 1):
        c = Case(fnpf, *shape, opts=fnpf.default_opts(rtol=1e-13, precond=pre, store_metric=store, max_iter=20000))
        phi = torch.zeros(c.om.N, dtype=torch.float64, device=c.dev)
        assert c.gm.laplace_solve(c.t(c.eta), c.t(c.phis), phi)["status"] == 0
        sol.append(phi.cpu().numpy())
    assert rel_l2(sol[1], sol[0]) < 1e-12
    phi_ref = osolve.laplace_solve(c.om, c.eta, c.h, c.phis)
    assert rel_l2(sol[1], phi_ref) < 1e-10


def _precond(c, fnpf, r, **kw):
    c.gm.set_opts(pmg(fnpf, **kw))
    z = torch.zeros_like(r)
    c.gm.profile_read(reset=True)
    c.gm.precond_apply(c.t(c.eta), r, z)
    torch.cuda.synchronize()
    return z, c.gm.profile_read(reset=True)["launches"]


@pytest.mark.parametrize("shape", [SHAPES[0], SHAPES[1], SHAPES[3], SHAPES[4], SHAPES[6], SHAPES[9],
                                   (3, 32, 32, 2, 6, True, True),
                                   (3, 96, 72, 2, 2, True, True),      # 13,824 coarse rows: 2 per thread
                                   (3, 60, 50, 3, 2, False, False)],   # 9,333 coarse rows, walls
                         ids=ids)
@pytest.mark.parametrize("coarse", [6, 31])
def test_cluster_coarse_solve_matches_per_step_launches(fnpf, shape, coarse):
    """The coarsest level's Chebyshev sweep on one thread-block cluster (stencil
    assembled from the level metric) applies the same polynomial as the
    per-step operator launches: the V-cycles agree to rounding, in far fewer
    launches."""
    c = Case(fnpf, *shape)
    r = torch.as_tensor(c.rng.standard_normal(c.gm.N - c.gm.ns), device=c.dev)
    zl, nl = _precond(c, fnpf, r, coarse_iters=coarse, coarse_solver=fnpf.FNPF_COARSE_LAUNCHES)
    zc, nc = _precond(c, fnpf, r, coarse_iters=coarse, coarse_solver=fnpf.FNPF_COARSE_CLUSTER)
    assert nc < nl, (nc, nl)
    assert rel_l2(zc.cpu().numpy(), zl.cpu().numpy()) < 1e-11


@pytest.mark.parametrize("shape", [SHAPES[0], SHAPES[3], SHAPES[4], SHAPES[7]], ids=ids)
@pytest.mark.parametrize("coarse_solver,kind", [("cluster", 1), ("launches", 1), ("cluster", 4), ("launches", 4)])
def test_pmg_preconditioner_is_symmetric_positive_definite(fnpf, shape, coarse_solver, kind):
    """PCG needs a fixed SPD preconditioner: <M r1, r2> = <r1, M r2> to
    rounding and <M r, r> > 0 (symmetric V-cycle, restriction = prolongation^T,
    polynomial smoothers of either kind, symmetric coarse stencil)."""
    c = Case(fnpf, *shape)
    mode = fnpf.FNPF_COARSE_CLUSTER if coarse_solver == "cluster" else fnpf.FNPF_COARSE_LAUNCHES
    n = c.gm.N - c.gm.ns
    r1 = torch.as_tensor(c.rng.standard_normal(n), device=c.dev)
    r2 = torch.as_tensor(c.rng.standard_normal(n), device=c.dev)
    z1, _ = _precond(c, fnpf, r1, coarse_solver=mode, cheb_kind=kind)
    z2, _ = _precond(c, fnpf, r2, coarse_solver=mode, cheb_kind=kind)
    a, b = float(torch.dot(z1, r2)), float(torch.dot(r1, z2))
    scale = float(torch.linalg.norm(z1) * torch.linalg.norm(r2))
    assert abs(a - b) < 1e-12 * scale, (a, b)
    assert float(torch.dot(z1, r1)) > 0 and float(torch.dot(z2, r2)) > 0


def test_jacobi_preconditioner_apply_is_inverse_diagonal(fnpf):
    c = Case(fnpf, *SHAPES[3])
    c.gm.set_opts(fnpf.default_opts())
    n = c.gm.N - c.gm.ns
    r = torch.as_tensor(c.rng.standard_normal(n), device=c.dev)
    z = torch.zeros_like(r)
    d = torch.zeros(c.gm.N, dtype=torch.float64, device=c.dev)
    c.gm.precond_apply(c.t(c.eta), r, z)
    c.gm.diagonal(c.t(c.eta), d)
    torch.cuda.synchronize()
    assert rel_l2(z.cpu().numpy(), (r / d[:n]).cpu().numpy()) < 1e-15


@pytest.mark.parametrize("shape", [SHAPES[0], SHAPES[1], SHAPES[3], SHAPES[5], SHAPES[7]], ids=ids)
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_fourth_kind_smoother_solve_matches_oracle(fnpf, shape, precision):
    prec = fnpf.FNPF_MIXED if precision == "mixed" else fnpf.FNPF_FP64
    c = Case(fnpf, *shape, opts=pmg(fnpf, precision=prec, cheb_kind=fnpf.FNPF_CHEB_FOURTH, inner_rtol=1e-5))
    phi_ref = osolve.laplace_solve(c.om, c.eta, c.h, c.phis)
    phi = torch.zeros(c.om.N, dtype=torch.float64, device=c.dev)
    info = c.gm.laplace_solve(c.t(c.eta), c.t(c.phis), phi)
    assert info["status"] == 0 and info["rel_res"] <= 1e-13
    assert rel_l2(phi.cpu().numpy(), phi_ref) < 1e-10


def test_fourth_kind_one_step_is_scaled_jacobi(fnpf):
    """A p = 1 mesh has one multigrid level, so M is the coarse sweep alone; of
    degree 1 it is 4/(3 rho) D^-1 (fourth kind) or D^-1 / theta (first kind):
    z / (D^-1 r) is one constant, and rho = 4 / (3 const) is the same as the
    first kind's lmax = 2 theta / (1 + 1/20)."""
    c = Case(fnpf, *SHAPES[7])
    n = c.gm.N - c.gm.ns
    r = torch.as_tensor(c.rng.standard_normal(n), device=c.dev)
    d = torch.zeros(c.gm.N, dtype=torch.float64, device=c.dev)
    c.gm.diagonal(c.t(c.eta), d)
    ratios = []
    for kind in (fnpf.FNPF_CHEB_FOURTH, fnpf.FNPF_CHEB_FIRST):
        z, _ = _precond(c, fnpf, r, coarse_iters=1, cheb_kind=kind)
        q = (z * d[:n] / r).cpu().numpy()
        assert np.ptp(q) < 1e-12 * abs(q.mean())
        ratios.append(q.mean())
    rho4 = 4.0 / (3.0 * ratios[0])
    rho1 = 2.0 / (ratios[1] * (1.0 + 1.0 / fnpf.default_opts().cheb_range))
    assert abs(rho4 - rho1) < 1e-10 * rho1 and 1.0 < rho4 < 20.0


@pytest.mark.parametrize("shape", [SHAPES[0], SHAPES[1], SHAPES[3], SHAPES[4], SHAPES[5]], ids=ids)
@pytest.mark.parametrize("schedule", ["two", "step2"])
def test_level_schedules_solve_and_stay_spd(fnpf, shape, schedule):
    """The two-level (p -> 1) and steps-of-two (p -> p-2 -> ... -> 1) level
    sequences give the oracle's solution and a symmetric positive definite
    V-cycle."""
    sched = fnpf.FNPF_MG_TWO_LEVEL if schedule == "two" else fnpf.FNPF_MG_STEP2
    c = Case(fnpf, *shape, opts=pmg(fnpf, mg_schedule=sched))
    phi_ref = osolve.laplace_solve(c.om, c.eta, c.h, c.phis)
    phi = torch.zeros(c.om.N, dtype=torch.float64, device=c.dev)
    info = c.gm.laplace_solve(c.t(c.eta), c.t(c.phis), phi)
    assert info["status"] == 0 and rel_l2(phi.cpu().numpy(), phi_ref) < 1e-10
    n = c.gm.N - c.gm.ns
    r1 = torch.as_tensor(c.rng.standard_normal(n), device=c.dev)
    r2 = torch.as_tensor(c.rng.standard_normal(n), device=c.dev)
    z1, _ = _precond(c, fnpf, r1, mg_schedule=sched)
    z2, _ = _precond(c, fnpf, r2, mg_schedule=sched)
    a, b = float(torch.dot(z1, r2)), float(torch.dot(r1, z2))
    assert abs(a - b) < 1e-12 * float(torch.linalg.norm(z1) * torch.linalg.norm(r2))
    assert float(torch.dot(z1, r1)) > 0


@pytest.mark.parametrize("shape", [SHAPES[0], SHAPES[1], SHAPES[3], SHAPES[4], SHAPES[6]], ids=ids)
def test_fp64_pcg_with_fp32_multigrid_matches_oracle(fnpf, shape):
    """FNPF_FP64_PC32: FP64 PCG (FP64 operator, residuals, dots) with the
    p-multigrid V-cycle in FP32 reaches the oracle's solution at rtol 1e-13."""
    c = Case(fnpf, *shape, opts=pmg(fnpf, precision=fnpf.FNPF_FP64_PC32))
    phi_ref = osolve.laplace_solve(c.om, c.eta, c.h, c.phis)
    phi = torch.zeros(c.om.N, dtype=torch.float64, device=c.dev)
    info = c.gm.laplace_solve(c.t(c.eta), c.t(c.phis), phi)
    assert info["status"] == 0 and info["rel_res"] <= 1e-13
    assert rel_l2(phi.cpu().numpy(), phi_ref) < 1e-10


@pytest.mark.parametrize("model", ["fnpf", "lpf"])
def test_fp64_pc32_rk4_steps_match_oracle(fnpf, model):
    """Host-driven and graph-replayed RK4 steps with the FP32 preconditioner."""
    lin = model == "lpf"
    c = Case(fnpf, 3, 5, 3, 2, 5, True, False,
             opts=pmg(fnpf, precision=fnpf.FNPF_FP64_PC32, model=fnpf.FNPF_LINEAR if lin else fnpf.FNPF_NONLINEAR))
    dt = 0.01
    eta_r, phi_r = c.eta.copy(), c.phis.copy()
    eta, phis = c.t(c.eta), c.t(c.phis)
    for n in range(4):
        eta_r, phi_r = osurf.rk4_step(c.om, c.h, eta_r, phi_r, dt, 9.81, linear=lin)
        c.gm.rk4_step(eta, phis, n * dt, dt)
    torch.cuda.synchronize()
    assert rel_l2(eta.cpu().numpy(), eta_r) < 1e-10
    assert rel_l2(phis.cpu().numpy(), phi_r) < 1e-10
