"""Adjoint of the RK4 step (hand-written reverse mode with one adjoint Laplace
solve per stage) against the oracle's exact tangent-linear model (complex
step) through the dot-product identity <lam, J d> = <J^T lam, d>, and the
checkpointed multi-step gradient against central finite differences,
including the gradient with respect to a bottom-bump amplitude."""
import math

import numpy as np
import pytest
import torch

from oracle import mesh as omesh
from oracle import tlm
from paper_2506_09435_gb300 import workloads as W
from paper_2506_09435_gb300.autograd import rk4_run
from tests.pairs import Case

pytestmark = pytest.mark.gpu


def adjoint_dot_test(fnpf, c, h, dt, relax=None):
    rng = np.random.default_rng(11)
    le, lp, de, dp, dh = (rng.standard_normal(c.om.ns) for _ in range(5))
    te, tp = tlm.step_tlm(c.om, h, c.eta, c.phis, dt, 9.81, de, dp, dh, relax=relax)
    lhs = le @ te + lp @ tp
    oe, op_ = torch.empty_like(c.t(le)), torch.empty_like(c.t(lp))
    lh = torch.zeros_like(oe)
    c.gm.step_adjoint(c.t(c.eta), c.t(c.phis), c.t(le), c.t(lp), oe, op_, lh, 0.0, dt)
    torch.cuda.synchronize()
    rhs = oe.cpu().numpy() @ de + op_.cpu().numpy() @ dp + lh.cpu().numpy() @ dh
    return lhs, rhs


@pytest.mark.parametrize("shape", [(3, 3, 2, 2, 3, True, False), (3, 4, 3, 2, 4, False, False),
                                   (2, 6, 1, 2, 4, True, False), (3, 3, 3, 1, 5, True, True)],
                         ids=["3d_PW_p3", "3d_WW_p4", "2d_p4", "3d_PP_p5"])
@pytest.mark.parametrize("precond", ["jacobi", "pmg"])
def test_adjoint_dot_product_with_oracle_tlm(fnpf, shape, precond):
    pre = fnpf.FNPF_PMG if precond == "pmg" else fnpf.FNPF_JACOBI
    c = Case(fnpf, *shape, amp=0.05, hvar=0.15, opts=fnpf.default_opts(rtol=1e-13, precond=pre, max_iter=50000))
    lhs, rhs = adjoint_dot_test(fnpf, c, c.h, 0.02)
    assert abs(lhs - rhs) <= 1e-9 * abs(lhs), (lhs, rhs)


def test_adjoint_with_relaxation_zones(fnpf):
    d = W.bar_flume(nx=8, ny=2, nz=2, p=3, Lx=8.0)
    d["zone"] = 2.0
    c = Case(fnpf, 3, 8, 2, 2, 3, False, False, Lx=8.0, Ly=d["Ly"], amp=0.02,
             opts=fnpf.default_opts(rtol=1e-13, max_iter=50000))
    cr, gen = W.flume_zones(d, c.x)
    wave = W.flume_wave(d)
    c.gm.set_relaxation(cr, gen, **wave)
    lhs, rhs = adjoint_dot_test(fnpf, c, c.h, d["T"] / 50, relax=(cr, gen, wave))
    assert abs(lhs - rhs) <= 1e-9 * abs(lhs), (lhs, rhs)


def test_checkpointed_gradient_matches_finite_differences(fnpf):
    """J = sum of c . eta after 5 steps (a weighted probe elevation); gradients
    with respect to the initial state (checkpoint every 2 steps) and to the
    amplitude A of a Gaussian bottom bump h = h0 - A exp(-r^2 / (2 s^2)), A = 0."""
    shape = (3, 4, 3, 2, 3, True, False)
    opts = fnpf.default_opts(rtol=1e-13, precond=fnpf.FNPF_PMG, max_iter=50000)
    c = Case(fnpf, *shape, amp=0.04, hvar=0.0, opts=opts)
    dev = c.dev
    x, y = c.x, c.y
    bump = np.exp(-((x - 0.5) ** 2 + (y - 0.4) ** 2) / (2 * 0.15 ** 2))
    probe = np.exp(-((x - 0.3) ** 2 + (y - 0.6) ** 2) / (2 * 0.1 ** 2))
    dt, nsteps = 0.02, 5
    eta0 = c.t(c.eta).requires_grad_(True)
    phi0 = c.t(c.phis).requires_grad_(True)
    h_t = c.t(c.h).requires_grad_(True)
    eN, pN = rk4_run(c.gm, eta0, phi0, h_t, 0.0, dt, nsteps, every=2)
    J = (eN * c.t(probe)).sum()
    J.backward()
    ge, gp, gh = eta0.grad.cpu().numpy(), phi0.grad.cpu().numpy(), h_t.grad.cpu().numpy()

    def run(eta, phis, h):
        gm = fnpf.Mesh(*shape[:5], shape[5], shape[6], h, g=9.81, opts=opts)
        e, p = c.t(eta), c.t(phis)
        for n in range(nsteps):
            gm.rk4_step(e, p, n * dt, dt)
        torch.cuda.synchronize()
        return float(e.cpu().numpy() @ probe)

    rng = np.random.default_rng(5)
    de, dp = rng.standard_normal(c.om.ns), rng.standard_normal(c.om.ns)
    s = 1e-6
    fd = (run(c.eta + s * de, c.phis + s * dp, c.h) - run(c.eta - s * de, c.phis - s * dp, c.h)) / (2 * s)
    ad = ge @ de + gp @ dp
    assert abs(fd - ad) <= 1e-6 * abs(ad), (fd, ad)
    sA = 1e-6
    fdA = (run(c.eta, c.phis, c.h - sA * bump) - run(c.eta, c.phis, c.h + sA * bump)) / (2 * sA)
    adA = -(gh @ bump)
    assert abs(fdA - adA) <= 1e-5 * abs(adA), (fdA, adA)


def test_taped_adjoint_equals_recomputing_adjoint(fnpf):
    """fnpf_step_adjoint_taped on the stage data recorded by fnpf_rk4_step
    (graph-replayed steps) gives fnpf_step_adjoint's result (which recomputes
    the step) to the solver tolerance, on every recorded step."""
    shape = (3, 4, 3, 2, 4, True, False)
    c = Case(fnpf, *shape, amp=0.05, opts=fnpf.default_opts(rtol=1e-13, precond=fnpf.FNPF_PMG, max_iter=50000))
    dt, nsteps = 0.02, 3
    eta, phis = c.t(c.eta), c.t(c.phis)
    c.gm.rk4_step(eta.clone(), phis.clone(), 0.0, dt)       # host-driven warm-up: the next steps replay graphs
    states = []
    c.gm.tape_begin(nsteps)
    for n in range(nsteps):
        states.append((eta.clone(), phis.clone()))
        c.gm.rk4_step(eta, phis, n * dt, dt)
    c.gm.tape_end()
    rng = np.random.default_rng(2)
    le, lp = c.t(rng.standard_normal(c.om.ns)), c.t(rng.standard_normal(c.om.ns))
    for n in range(nsteps):
        a = [torch.empty_like(le) for _ in range(2)] + [torch.zeros_like(le)]
        b = [torch.empty_like(le) for _ in range(2)] + [torch.zeros_like(le)]
        c.gm.step_adjoint(states[n][0], states[n][1], le, lp, a[0], a[1], a[2], n * dt, dt)
        c.gm.step_adjoint_taped(n, le, lp, b[0], b[1], b[2], dt)
        torch.cuda.synchronize()
        for x, y in zip(a, b):
            assert float(torch.linalg.norm(x - y) / torch.linalg.norm(x)) < 1e-10
    with pytest.raises(fnpf.FnpfError):
        c.gm.step_adjoint_taped(nsteps, le, lp, le.clone(), lp.clone(), None, dt)
