"""Element-wise parity with the FP64 oracle of the forms that wrap the plain
RK4 step: the batched ensemble (every tank against the oracle's own RK4
step), the adjoint step (the whole vector J^T lam, component by component,
against the oracle's complex-step tangent-linear model), and a tank of the
benchmark's element shape and order carried for 20 graph-replayed RK4 steps
with the p-multigrid solver in FP64 and in both mixed-precision forms.

Tolerances: relative L2 1e-10 for FP64 results (solves to rtol 1e-13, the
reading that parity runs solve well below the configurations' 1e-10), 1e-8
for the mixed-precision forms, 1e-9 (max norm) for the adjoint, whose
right-hand sides carry the adjoint solves' residuals."""
import os

import numpy as np
import pytest
import torch

from oracle import mesh as omesh
from oracle import surface as osurf
from oracle import tlm
from paper_2506_09435_gb300 import workloads as W
from tests.pairs import Case, rel_l2, rel_max

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))


# ----------------------------------------------------------------------------- ensemble

@pytest.mark.parametrize("prec,tol", [("fp64", 1e-10), ("mixed", 1e-8), ("pc32", 1e-10)])
def test_ensemble_tanks_match_oracle(fnpf, prec, tol):
    """Four periodic tanks of different element counts (nx != ny) and orders
    p = 6, 4, 3, 2, kh and steepness from the ensemble generator, advanced 3
    RK4 steps by fnpf_ensemble_rk4_step (steps 2 and 3 replay the ensemble's
    one captured graph); every tank equals the oracle's steps."""
    precision = {"fp64": fnpf.FNPF_FP64, "mixed": fnpf.FNPF_MIXED, "pc32": fnpf.FNPF_FP64_PC32}[prec]
    o = fnpf.default_opts(rtol=1e-13, precond=fnpf.FNPF_PMG, precision=precision, max_iter=50000)
    tanks = W.ensemble_tanks(n=4, seed=16, nmin=2, nmax=4, pmin=2, pmax=6)
    assert sorted(d["p"] for d in tanks) == [2, 3, 4, 6]
    dev = torch.device("cuda:0")
    meshes, oms, hs, etas, phiss, dts, refs = [], [], [], [], [], [], []
    for d in tanks:
        om = omesh.Mesh(3, d["nx"], d["ny"], 2, d["p"], True, True, d["Lx"], d["Ly"])
        x, y = om.surface_coords()
        h = np.full(om.ns, d["h0"])
        m = fnpf.Mesh(3, d["nx"], d["ny"], 2, d["p"], True, True, h, Lx=d["Lx"], Ly=d["Ly"], g=d["g"], opts=o)
        e0, p0 = W.airy_plus_spectrum_state(d, x, y, seed=d["seed"], steepness=d["steepness"])
        meshes.append(m)
        oms.append(om)
        hs.append(h)
        etas.append(torch.tensor(e0, dtype=torch.float64, device=dev))
        phiss.append(torch.tensor(p0, dtype=torch.float64, device=dev))
        dts.append(W.period(d["k"], d["h0"], d["g"]) / 100)
        refs.append((e0, p0))
    ens = fnpf.Ensemble(meshes)
    for k in range(3):
        infos = ens.rk4_step(etas, phiss, [k * dt for dt in dts], dts, info=True)
        assert all(i["status"] == 0 for i in infos)
    torch.cuda.synchronize()
    for i, d in enumerate(tanks):
        e_r, p_r = refs[i]
        for _ in range(3):
            e_r, p_r = osurf.rk4_step(oms[i], hs[i], e_r, p_r, dts[i], d["g"])
        assert rel_l2(etas[i].cpu().numpy(), e_r) < tol, (i, d["p"])
        assert rel_l2(phiss[i].cpu().numpy(), p_r) < tol, (i, d["p"])


# ----------------------------------------------------------------------------- adjoint

@pytest.mark.parametrize("shape,precond", [((3, 3, 2, 1, 2, True, False), "jacobi"),
                                           ((3, 2, 2, 2, 3, True, True), "pmg"),
                                           ((2, 4, 1, 2, 3, True, False), "pmg")],
                         ids=["3d_PW_p2_jacobi", "3d_PP_p3_pmg", "2d_p3_pmg"])
def test_adjoint_vector_matches_oracle_tlm_componentwise(fnpf, shape, precond):
    """J^T lam of one RK4 step, for J = d(eta_{n+1}, phi_{n+1}) / d(eta_n,
    phi_n, h), assembled from the oracle's exact directional derivatives (one
    complex-step run per unit perturbation of each eta_n, phi_n and h node),
    against fnpf_step_adjoint's lam_eta_out, lam_phis_out and lam_h."""
    pre = fnpf.FNPF_PMG if precond == "pmg" else fnpf.FNPF_JACOBI
    c = Case(fnpf, *shape, amp=0.05, hvar=0.15, opts=fnpf.default_opts(rtol=1e-13, precond=pre, max_iter=50000))
    ns, dt, g = c.om.ns, 0.02, 9.81
    assert ns <= 60
    rng = np.random.default_rng(3)
    le, lp = rng.standard_normal(ns), rng.standard_normal(ns)
    ref = np.zeros((3, ns))
    zero = np.zeros(ns)
    for i in range(ns):
        unit = np.zeros(ns)
        unit[i] = 1.0
        for a, (de, dp, dh) in enumerate(((unit, zero, zero), (zero, unit, zero), (zero, zero, unit))):
            te, tp = tlm.step_tlm(c.om, c.h, c.eta, c.phis, dt, g, de, dp, dh)
            ref[a, i] = le @ te + lp @ tp
    oe, op_ = torch.empty(ns, dtype=torch.float64, device=c.dev), torch.empty(ns, dtype=torch.float64, device=c.dev)
    lh = torch.zeros_like(oe)
    c.gm.step_adjoint(c.t(c.eta), c.t(c.phis), c.t(le), c.t(lp), oe, op_, lh, 0.0, dt)
    torch.cuda.synchronize()
    got = np.stack([oe.cpu().numpy(), op_.cpu().numpy(), lh.cpu().numpy()])
    for a, name in enumerate(("lam_eta", "lam_phis", "lam_h")):
        assert rel_max(got[a], ref[a]) < 1e-9, (name, rel_max(got[a], ref[a]))


# ----------------------------------------------------------------------------- 20 steps, p = 6

def _box_p6_trajectory():
    path = os.path.join(HERE, "golden", "box_p6_8x8x2_trajectory.npz")
    return np.load(path)


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-10), ("pc32", 1e-10), ("mixed", 1e-8)])
def test_p6_tank_20_graph_replayed_steps_match_oracle(fnpf, prec, tol):
    """The benchmark tank's element shape and order (p = 6, 2 layers, kh = 2,
    Airy wave plus the seeded spectrum, dt = T/100) on 8 x 8 columns of
    elements, p-multigrid PCG, 20 RK4 steps (steps 2-20 replay one captured
    graph each) against the oracle's trajectory stored by
    tests/golden/make_box_p6_trajectory.py."""
    ref = _box_p6_trajectory()
    precision = {"fp64": fnpf.FNPF_FP64, "mixed": fnpf.FNPF_MIXED, "pc32": fnpf.FNPF_FP64_PC32}[prec]
    d = W.periodic_box_3d(nx=8, ny=8, nz=2, p=6, kh=2.0)
    o = fnpf.default_opts(rtol=1e-13, precond=fnpf.FNPF_PMG, precision=precision, max_iter=50000)
    m = fnpf.Mesh(3, 8, 8, 2, 6, True, True, ref["h"], Lx=d["Lx"], Ly=d["Ly"], g=d["g"], opts=o)
    dev = torch.device("cuda:0")
    eta = torch.tensor(ref["eta0"], dtype=torch.float64, device=dev)
    phis = torch.tensor(ref["phis0"], dtype=torch.float64, device=dev)
    dt = float(ref["dt"])
    for n in range(20):
        infos = m.rk4_step(eta, phis, n * dt, dt, info=True)
        assert all(i["status"] == 0 for i in infos)
        if n == 0:
            torch.cuda.synchronize()
            assert rel_l2(eta.cpu().numpy(), ref["eta1"]) < tol
            assert rel_l2(phis.cpu().numpy(), ref["phis1"]) < tol
    torch.cuda.synchronize()
    e20, p20 = eta.cpu().numpy(), phis.cpu().numpy()
    assert rel_l2(e20, ref["eta20"]) < tol, rel_l2(e20, ref["eta20"])
    assert rel_l2(p20, ref["phis20"]) < tol, rel_l2(p20, ref["phis20"])


# ----------------------------------------------------------------------------- invariants

@pytest.mark.parametrize("shape", [(3, 4, 3, 2, 4, True, False), (3, 3, 3, 2, 5, False, False),
                                   (2, 6, 1, 2, 4, True, False)], ids=["3d_PW_p4", "3d_WW_p5", "2d_p4"])
def test_invariants_match_oracle(fnpf, shape):
    """fnpf_invariants (mass and energy of the state) against the oracle's
    surface.mass and surface.energy on the same curved, variable-depth mesh."""
    c = Case(fnpf, *shape, amp=0.05, hvar=0.15, opts=fnpf.default_opts(rtol=1e-13, max_iter=50000))
    m_gpu, e_gpu = c.gm.invariants(c.t(c.eta), c.t(c.phis))
    m_ref = osurf.mass(c.om, c.eta)
    e_ref = osurf.energy(c.om, c.h, c.eta, c.phis, 9.81)
    # the mass of a zero-mean wave is a sum of cancelling terms: bound by the scale of the terms
    scale = osurf.mass(c.om, np.abs(c.eta))
    assert abs(m_gpu - m_ref) <= 1e-13 * scale, (m_gpu, m_ref)
    assert abs(e_gpu - e_ref) <= 1e-10 * abs(e_ref), (e_gpu, e_ref)


# ----------------------------------------------------------------------------- initial-guess projection

def test_projected_initial_guess_keeps_results_and_saves_iterations(fnpf):
    """The Galerkin projection of the initial guess onto the last solutions
    (opts.projection) changes only where CG starts: RK4 states agree with the
    unprojected solver to the solve tolerance, match the oracle, and the
    solves of later steps need fewer iterations."""
    shape = (3, 4, 4, 2, 5, True, True)
    res = {}
    for L in (0, 8):
        o = fnpf.default_opts(rtol=1e-12, precond=fnpf.FNPF_PMG, projection=L)
        c = Case(fnpf, *shape, opts=o)
        eta, phis = c.t(c.eta), c.t(c.phis)
        iters = []
        for k in range(4):
            inf = c.gm.rk4_step(eta, phis, 0.01 * k, 0.01, info=True)
            iters.append(sum(i["iters"] for i in inf))
        torch.cuda.synchronize()
        res[L] = (eta.cpu().numpy(), phis.cpu().numpy(), iters)
    e_r, p_r = c.eta, c.phis
    for k in range(4):
        e_r, p_r = osurf.rk4_step(c.om, c.h, e_r, p_r, 0.01, 9.81)
    for L in (0, 8):
        assert rel_l2(res[L][0], e_r) < 1e-10 and rel_l2(res[L][1], p_r) < 1e-10
    assert rel_l2(res[8][0], res[0][0]) < 1e-11
    assert sum(res[8][2][1:]) < 0.8 * sum(res[0][2][1:]), (res[0][2], res[8][2])


def test_projection_keeps_an_exact_caller_guess(fnpf):
    """fnpf_laplace_solve with the caller's guess already the solution: the
    guess is a basis vector of the projection, so the solve starts converged
    whatever the history holds."""
    c = Case(fnpf, 3, 3, 3, 2, 4, True, False, opts=fnpf.default_opts(rtol=1e-12, precond=fnpf.FNPF_PMG))
    eta, phis = c.t(c.eta), c.t(c.phis)
    phi = torch.zeros(c.om.N, dtype=torch.float64, device=c.dev)
    c.gm.laplace_solve(eta, phis, phi)                       # fills the history
    c.gm.laplace_solve(eta, c.t(0.5 * c.phis), phi)          # a different solution in the history
    c.gm.laplace_solve(eta, phis, phi)
    exact = phi.clone()
    info = c.gm.laplace_solve(eta, phis, phi)
    assert info["iters"] <= 1, info
    torch.cuda.synchronize()
    assert rel_l2(phi.cpu().numpy(), exact.cpu().numpy()) < 1e-11
