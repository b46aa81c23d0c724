"""Mixed-precision form (FP32 operator and inner Jacobi-PCG, FP64 defect
correction, FP64 dot products): parity of the FP32 operator with the oracle at
FP32 accuracy, and of solves and RK4 states with the oracle / the FP64 path at
the FP64 tolerances (defect correction drives the FP64 residual to rtol)."""
import numpy as np
import pytest
import torch

from oracle import operator as oop
from oracle import solve as osolve
from oracle import surface as osurf
from tests.pairs import Case, rel_l2, rel_max

pytestmark = pytest.mark.gpu

SHAPES = [
    (2, 8, 1, 2, 4, True, False),
    (3, 5, 3, 2, 4, True, False),
    (3, 4, 4, 2, 6, True, True),
    (3, 3, 2, 3, 5, False, False),
]


def ids(s):
    return "d%d_%dx%dx%d_p%d" % s[:5]


def mixed(fnpf, rtol):
    return fnpf.default_opts(precision=fnpf.FNPF_MIXED, rtol=rtol, inner_rtol=1e-5, max_iter=50000)


@pytest.mark.parametrize("shape", SHAPES, ids=ids)
def test_fp32_operator_matches_oracle_to_fp32_accuracy(fnpf, shape):
    c = Case(fnpf, *shape)
    op = oop.Operator(c.om, c.eta, c.h)
    x = c.rng.standard_normal(c.om.N)
    y_ref = op.A @ x
    y = torch.empty(c.om.N, dtype=torch.float32, device=c.dev)
    c.gm.apply_f32(c.t(c.eta).float(), c.t(x).float(), y)
    torch.cuda.synchronize()
    assert rel_max(y.double().cpu().numpy(), y_ref) < 2e-6


@pytest.mark.parametrize("shape", SHAPES, ids=ids)
def test_mixed_solve_reaches_fp64_parity(fnpf, shape):
    c = Case(fnpf, *shape, opts=mixed(fnpf, 1e-13))
    phi_ref = osolve.laplace_solve(c.om, c.eta, c.h, c.phis)
    phi = torch.zeros(c.om.N, dtype=torch.float64, device=c.dev)
    info = c.gm.laplace_solve(c.t(c.eta), c.t(c.phis), phi)
    assert info["status"] == 0 and info["rel_res"] <= 1e-13 and info["outer_iters"] >= 1
    assert rel_l2(phi.cpu().numpy(), phi_ref) < 1e-10


@pytest.mark.parametrize("shape", [SHAPES[1], SHAPES[3]], ids=ids)
def test_mixed_rk4_matches_oracle_and_fp64_path(fnpf, shape):
    cm = Case(fnpf, *shape, opts=mixed(fnpf, 1e-10))
    cd = Case(fnpf, *shape, opts=fnpf.default_opts(rtol=1e-10))
    dt = 0.01
    eta_r, phi_r = cm.eta.copy(), cm.phis.copy()
    em, pm = cm.t(cm.eta), cm.t(cm.phis)
    ed, pd = cd.t(cd.eta), cd.t(cd.phis)
    for _ in range(3):
        eta_r, phi_r = osurf.rk4_step(cm.om, cm.h, eta_r, phi_r, dt, 9.81)
        cm.gm.rk4_step(em, pm, 0.0, dt)
        cd.gm.rk4_step(ed, pd, 0.0, dt)
    torch.cuda.synchronize()
    for a, b in [(em, ed), (pm, pd)]:
        assert rel_l2(a.cpu().numpy(), b.cpu().numpy()) < 1e-8
    assert rel_l2(em.cpu().numpy(), eta_r) < 1e-8
    assert rel_l2(pm.cpu().numpy(), phi_r) < 1e-8
