"""Isoparametric horizontal mesh (O-grid annulus around a vertical cylinder,
the shape of the cylinder case): operator, diagonal, solve, DtN/RHS, RK4 and
adjoint parity with the oracle, whose element Jacobians come from the same
nodal X, Y by its own general-inverse path."""
import numpy as np
import pytest
import torch

from oracle import mesh as omesh
from oracle import operator as oop
from oracle import solve as osolve
from oracle import surface as osurf
from oracle import tlm
from paper_2506_09435_gb300 import workloads as W
from tests.pairs import rel_l2, rel_max

pytestmark = pytest.mark.gpu


def ogrid(fnpf, nth=8, nr=3, nz=2, p=4, opts=None):
    d = W.cylinder_case(nth=nth, nr=nr, nz=nz, p=p, Rout=4.0)
    box = omesh.Mesh(3, nth, nr, nz, p, periodic_x=True, periodic_y=False, Lx=d["Lx"], Ly=d["Ly"])
    th, s = box.surface_coords()
    X, Y = W.ogrid_map(th, s, a=d["a"], R=d["R"])
    om = omesh.Mesh(3, nth, nr, nz, p, periodic_x=True, periodic_y=False, X=X, Y=Y)
    r = np.hypot(X, Y)
    h = d["h0"] * (1 + 0.1 * np.sin(0.5 * r) * np.cos(th))
    eta = 0.03 * d["h0"] * np.cos(d["k"] * X + 0.2) * np.exp(-0.05 * r)
    phis = 0.05 * np.sin(d["k"] * X) * np.cos(0.3 * Y)
    gm = fnpf.Mesh(3, nth, nr, nz, p, True, False, h, X=X, Y=Y, g=9.81,
                   opts=opts or fnpf.default_opts(rtol=1e-13, max_iter=50000))
    gx, gy = gm.surface_coords()
    assert np.max(np.abs(gx - X)) < 1e-13 and np.max(np.abs(gy - Y)) < 1e-13
    return om, gm, h, eta, phis


def T(a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device=torch.device("cuda:0"))


@pytest.mark.parametrize("p", [2, 4, 5])
def test_iso_operator_and_diagonal(fnpf, p):
    om, gm, h, eta, phis = ogrid(fnpf, p=p)
    op = oop.Operator(om, eta, h)
    x = np.random.default_rng(1).standard_normal(om.N)
    y = torch.empty(om.N, dtype=torch.float64, device="cuda:0")
    gm.apply(T(eta), T(x), y)
    d = torch.empty_like(y)
    gm.diagonal(T(eta), d)
    torch.cuda.synchronize()
    assert rel_max(y.cpu().numpy(), op.A @ x) < 1e-12
    assert rel_max(d.cpu().numpy(), op.A.diagonal()) < 1e-12


@pytest.mark.parametrize("precond", ["jacobi", "pmg"])
def test_iso_solve_dtn_rhs_rk4(fnpf, precond):
    pre = fnpf.FNPF_PMG if precond == "pmg" else fnpf.FNPF_JACOBI
    om, gm, h, eta, phis = ogrid(fnpf, opts=fnpf.default_opts(rtol=1e-13, precond=pre, max_iter=50000))
    w_ref, phi_ref = osolve.dtn(om, eta, h, phis)
    w = torch.empty(om.ns, dtype=torch.float64, device="cuda:0")
    gm.dtn(T(eta), T(phis), w)
    assert rel_l2(w.cpu().numpy(), w_ref) < 1e-10
    de_r, dp_r = osurf.zakharov_rhs(om, eta, phis, w_ref, 9.81)
    de, dp = torch.empty_like(w), torch.empty_like(w)
    gm.zakharov_rhs(T(eta), T(phis), T(w_ref), de, dp)
    torch.cuda.synchronize()
    assert rel_max(de.cpu().numpy(), de_r) < 1e-12 and rel_max(dp.cpu().numpy(), dp_r) < 1e-12
    e, p = T(eta), T(phis)
    er, pr = eta.copy(), phis.copy()
    for _ in range(2):
        er, pr = osurf.rk4_step(om, h, er, pr, 0.05, 9.81)
        gm.rk4_step(e, p, 0.0, 0.05)
    torch.cuda.synchronize()
    assert rel_l2(e.cpu().numpy(), er) < 1e-10 and rel_l2(p.cpu().numpy(), pr) < 1e-10


def test_iso_adjoint_dot_product(fnpf):
    om, gm, h, eta, phis = ogrid(fnpf, p=3)
    rng = np.random.default_rng(2)
    le, lp, de, dp, dh = (rng.standard_normal(om.ns) for _ in range(5))
    te, tp = tlm.step_tlm(om, h, eta, phis, 0.05, 9.81, de, dp, dh)
    oe, op_ = torch.empty(om.ns, dtype=torch.float64, device="cuda:0"), torch.empty(om.ns, dtype=torch.float64,
                                                                                     device="cuda:0")
    lh = torch.zeros_like(oe)
    gm.step_adjoint(T(eta), T(phis), T(le), T(lp), oe, op_, lh, 0.0, 0.05)
    torch.cuda.synchronize()
    lhs = le @ te + lp @ tp
    rhs = oe.cpu().numpy() @ de + op_.cpu().numpy() @ dp + lh.cpu().numpy() @ dh
    assert abs(lhs - rhs) <= 1e-9 * abs(lhs), (lhs, rhs)
