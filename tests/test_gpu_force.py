"""Gradients of the cylinder-force objective (configuration 4; paper
Sec. 3.2 around the RK4 step): the vector-Jacobian product of the Laplace
solve (fnpf_laplace_solve_vjp) against the oracle's complex-step derivative of
its solve, and the gradient of J = int F_x dt over a window of a short run
with respect to the initial state and a bottom-bump amplitude against the
oracle's complex-step tangent-linear model and central finite differences."""
import math

import numpy as np
import pytest
import torch

from oracle import mesh as omesh
from oracle import solve as osolve
from oracle import wall
from paper_2506_09435_gb300 import workloads as W

pytestmark = pytest.mark.gpu

NTH, NR, NZ, P = 8, 2, 2, 3


def ogrid(fnpf, h, opts):
    box = omesh.Mesh(3, NTH, NR, NZ, P, periodic_x=True, periodic_y=False, Lx=2 * math.pi, Ly=1.0)
    th, s = box.surface_coords()
    X, Y = W.ogrid_map(th, s, a=1.0, R=3.0)
    om = omesh.Mesh(3, NTH, NR, NZ, P, periodic_x=True, periodic_y=False, X=X, Y=Y)
    hh = h(X, Y) if callable(h) else h
    gm = fnpf.Mesh(3, NTH, NR, NZ, P, True, False, hh, X=X, Y=Y, opts=opts)
    return om, gm, X, Y, hh


def test_laplace_solve_vjp_matches_oracle_complex_step(fnpf):
    opts = fnpf.default_opts(rtol=1e-13, precond=fnpf.FNPF_PMG, max_iter=50000)
    om, gm, X, Y, h = ogrid(fnpf, lambda X, Y: 1.0 + 0.1 * np.cos(X) * np.exp(-(Y - 1.5) ** 2), opts)
    eta = 0.04 * np.cos(X + 0.2)
    phis = 0.1 * np.sin(X) + 0.05 * np.cos(Y)
    dev = torch.device("cuda:0")
    t = lambda a: torch.tensor(a, dtype=torch.float64, device=dev)
    phi = torch.zeros(om.N, dtype=torch.float64, device=dev)
    gm.laplace_solve(t(eta), t(phis), phi)
    rng = np.random.default_rng(3)
    gbar = rng.standard_normal(om.N)
    le, lp, lh = (torch.zeros(om.ns, dtype=torch.float64, device=dev) for _ in range(3))
    gm.laplace_solve_vjp(t(eta), t(phis), phi, t(gbar), le, lp, lh)
    torch.cuda.synchronize()
    de, dp, dh = rng.standard_normal(om.ns), rng.standard_normal(om.ns), rng.standard_normal(om.ns)
    eps = 1e-30
    ph_c = osolve.laplace_solve(om, eta + 1j * eps * de, h + 1j * eps * dh, phis + 1j * eps * dp)
    lhs = gbar @ (np.imag(ph_c) / eps)
    rhs = le.cpu().numpy() @ de + lp.cpu().numpy() @ dp + lh.cpu().numpy() @ dh
    assert abs(lhs - rhs) <= 1e-9 * abs(lhs), (lhs, rhs)


def test_force_gradient_matches_oracle_tlm_and_finite_differences(fnpf):
    from paper_2506_09435_gb300.objectives import WallForce, cylinder_force_objective
    opts = fnpf.default_opts(rtol=1e-13, precond=fnpf.FNPF_PMG, max_iter=50000)
    bump = lambda X, Y: np.exp(-((X + 2.0) ** 2 + Y ** 2) / 0.5)
    om, gm, X, Y, h = ogrid(fnpf, np.full(NTH * P * (NR * P + 1), 1.0), opts)
    k = 1.0
    om_ = 2 * math.pi / W.period(k, 1.0)
    eta0 = 0.02 * np.cos(k * X)
    phi0 = 9.81 * 0.02 / om_ * np.cosh(k * (eta0 + h)) / np.cosh(k * h) * np.sin(k * X)
    dt, n_a, n_b, g = 0.05, 2, 4, 9.81
    dev = torch.device("cuda:0")
    wf = WallForce(gm, X, Y, Mz=P + 2)
    e0 = torch.tensor(eta0, dtype=torch.float64, device=dev, requires_grad=True)
    p0 = torch.tensor(phi0, dtype=torch.float64, device=dev, requires_grad=True)
    ht = torch.tensor(h, dtype=torch.float64, device=dev, requires_grad=True)
    J = cylinder_force_objective(gm, wf, e0, p0, ht, 0.0, dt, n_a, n_b, every=2)
    J.backward()
    ge, gp, gh = e0.grad.cpu().numpy(), p0.grad.cpu().numpy(), ht.grad.cpu().numpy()
    J_ref = wall.force_integral(om, h, eta0, phi0, dt, g, n_a, n_b, Mz=P + 2)
    Jv = float(J.detach())
    assert abs(Jv - J_ref) <= 1e-9 * abs(J_ref), (Jv, J_ref)
    # oracle tangent-linear model (complex step) in a random direction of the state and the bump
    rng = np.random.default_rng(9)
    de, dp = rng.standard_normal(om.ns), rng.standard_normal(om.ns)
    bmp = bump(X, Y)
    eps = 1e-30
    Jc = wall.force_integral(om, h - 1j * eps * bmp, eta0 + 1j * eps * de, phi0 + 1j * eps * dp, dt, g, n_a, n_b,
                             Mz=P + 2)
    tlm = np.imag(Jc) / eps
    ad = ge @ de + gp @ dp - gh @ bmp
    assert abs(ad - tlm) <= 1e-8 * abs(tlm), (ad, tlm)
    # central differences of the GPU forward in the state direction
    def run(eta, phis, hh):
        m2 = fnpf.Mesh(3, NTH, NR, NZ, P, True, False, hh, X=X, Y=Y, opts=opts)
        w2 = WallForce(m2, X, Y, Mz=P + 2)
        with torch.no_grad():
            return float(cylinder_force_objective(m2, w2, torch.tensor(eta, dtype=torch.float64, device=dev),
                                                  torch.tensor(phis, dtype=torch.float64, device=dev),
                                                  torch.tensor(hh, dtype=torch.float64, device=dev), 0.0, dt,
                                                  n_a, n_b, every=2))
    s = 1e-6
    fd = (run(eta0 + s * de, phi0 + s * dp, h) - run(eta0 - s * de, phi0 - s * dp, h)) / (2 * s)
    assert abs(fd - (ge @ de + gp @ dp)) <= 1e-6 * abs(fd), (fd, ge @ de + gp @ dp)
