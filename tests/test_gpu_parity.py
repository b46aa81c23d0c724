"""Parity of the CUDA path with the FP64 oracle on the same seeded inputs
(operator, Jacobi diagonal, Laplace solve, DtN map, Zakharov RHS, RK4).

Tolerances: operator and diagonal agree to rounding (<= 1e-12 relative to the
largest entry); solves, DtN and RK4 states to <= 1e-10 relative L2, the FP64
bound of the method (solver rtol 1e-13 here, so the algebraic error stays
below it)."""
import math

import numpy as np
import pytest
import torch

from oracle import operator as oop
from oracle import solve as osolve
from oracle import surface as osurf
from paper_2506_09435_gb300 import workloads
from tests.pairs import Case, rel_l2, rel_max

pytestmark = pytest.mark.gpu

# (dim, nx, ny, nz, p, periodic_x, periodic_y): several CTAs and ragged tails
SHAPES = [
    (2, 8, 1, 2, 4, True, False),
    (2, 5, 1, 3, 7, False, False),
    (3, 5, 3, 2, 4, True, False),
    (3, 4, 4, 2, 6, True, True),
    (3, 3, 2, 3, 5, False, False),
    (3, 2, 3, 1, 8, False, True),
    (3, 7, 3, 2, 2, True, True),
    (3, 3, 2, 2, 1, True, False),
    (3, 2, 2, 1, 3, True, True),
    (3, 5, 2, 2, 3, False, True),
]


def ids(s):
    return "d%d_%dx%dx%d_p%d_%s%s" % (s[0], s[1], s[2], s[3], s[4], "P" if s[5] else "W", "P" if s[6] else "W")


@pytest.mark.parametrize("shape", SHAPES, ids=ids)
def test_apply_matches_oracle(fnpf, shape):
    c = Case(fnpf, *shape)
    op = oop.Operator(c.om, c.eta, c.h)
    for trial in range(2):
        x = c.rng.standard_normal(c.om.N)
        y_ref = op.A @ x
        y = torch.empty(c.om.N, dtype=torch.float64, device=c.dev)
        c.gm.apply(c.t(c.eta), c.t(x), y)
        torch.cuda.synchronize()
        assert rel_max(y.cpu().numpy(), y_ref) < 1e-12


@pytest.mark.parametrize("shape", SHAPES, ids=ids)
def test_diagonal_matches_oracle(fnpf, shape):
    c = Case(fnpf, *shape)
    d_ref = oop.Operator(c.om, c.eta, c.h).A.diagonal()
    d = torch.empty(c.om.N, dtype=torch.float64, device=c.dev)
    c.gm.diagonal(c.t(c.eta), d)
    torch.cuda.synchronize()
    assert rel_max(d.cpu().numpy(), d_ref) < 1e-12


def tight(fnpf):
    return fnpf.default_opts(rtol=1e-13, max_iter=50000)


@pytest.mark.parametrize("shape", SHAPES, ids=ids)
def test_laplace_solve_matches_oracle(fnpf, shape):
    c = Case(fnpf, *shape, opts=tight(fnpf))
    phi_ref = osolve.laplace_solve(c.om, c.eta, c.h, c.phis)
    phi = torch.zeros(c.om.N, dtype=torch.float64, device=c.dev)
    info = c.gm.laplace_solve(c.t(c.eta), c.t(c.phis), phi)
    assert info["status"] == 0 and info["rel_res"] <= 1e-13
    assert rel_l2(phi.cpu().numpy(), phi_ref) < 1e-10
    # warm start from the solution converges at once and stays put
    info2 = c.gm.laplace_solve(c.t(c.eta), c.t(c.phis), phi)
    assert info2["iters"] <= 1
    assert rel_l2(phi.cpu().numpy(), phi_ref) < 1e-10


@pytest.mark.parametrize("shape", SHAPES, ids=ids)
def test_dtn_and_rhs_match_oracle(fnpf, shape):
    c = Case(fnpf, *shape, opts=tight(fnpf))
    w_ref, _ = osolve.dtn(c.om, c.eta, c.h, c.phis)
    w = torch.zeros(c.om.ns, dtype=torch.float64, device=c.dev)
    c.gm.dtn(c.t(c.eta), c.t(c.phis), w)
    assert rel_l2(w.cpu().numpy(), w_ref) < 1e-10
    # right-hand side from the same w on both sides
    de_ref, dp_ref = osurf.zakharov_rhs(c.om, c.eta, c.phis, w_ref, 9.81)
    de = torch.empty_like(w)
    dp = torch.empty_like(w)
    c.gm.zakharov_rhs(c.t(c.eta), c.t(c.phis), c.t(w_ref), de, dp)
    torch.cuda.synchronize()
    assert rel_max(de.cpu().numpy(), de_ref) < 1e-12
    assert rel_max(dp.cpu().numpy(), dp_ref) < 1e-12


@pytest.mark.parametrize("shape", [SHAPES[0], SHAPES[2], SHAPES[4]], ids=ids)
def test_rk4_steps_match_oracle(fnpf, shape):
    c = Case(fnpf, *shape, opts=tight(fnpf))
    dt = 0.01
    eta_r, phi_r = c.eta.copy(), c.phis.copy()
    eta, phis = c.t(c.eta), c.t(c.phis)
    for _ in range(3):
        eta_r, phi_r = osurf.rk4_step(c.om, c.h, eta_r, phi_r, dt, 9.81)
        c.gm.rk4_step(eta, phis, 0.0, dt)
    torch.cuda.synchronize()
    assert rel_l2(eta.cpu().numpy(), eta_r) < 1e-10
    assert rel_l2(phis.cpu().numpy(), phi_r) < 1e-10


def test_standing_wave_2d_full_run_matches_oracle(fnpf):
    """The 2D 8 x 2, p = 4 standing-wave tank for 4 periods (256 RK4 steps,
    dt = T/64), Jacobi-PCG at rtol 1e-12 on the GPU against the oracle's
    direct solves.  At every step eta and phi_eta agree to 1e-10 relative to
    their amplitude over the run; where each field peaks (phi_eta at t = 3.75 T,
    eta at t = 4 T) also to 1e-10 in plain relative L2.  (At t = 4 T phi_eta is
    near a zero of its oscillation, so its plain relative error is not a
    meaningful measure there.)"""
    d = workloads.standing_wave_2d()
    c = Case(fnpf, 2, d["nx"], 1, d["nz"], d["p"], True, False, Lx=d["Lx"], h0=d["h0"], hvar=0.0,
             opts=fnpf.default_opts(rtol=1e-12))
    h = np.full(c.om.ns, d["h0"])
    eta0, phi0 = workloads.standing_wave_state(d, c.x)
    T = workloads.period(d["k"], d["h0"], d["g"])
    dt = T / 64
    eta_r, phi_r = eta0.copy(), phi0.copy()
    eta, phis = c.t(eta0), c.t(phi0)
    hist = []
    for n in range(256):
        eta_r, phi_r = osurf.rk4_step(c.om, h, eta_r, phi_r, dt, d["g"])
        c.gm.rk4_step(eta, phis, n * dt, dt)
        hist.append((eta.cpu().numpy(), phis.cpu().numpy(), eta_r.copy(), phi_r.copy()))
    amp_e = max(np.linalg.norm(hh[2]) for hh in hist)
    amp_p = max(np.linalg.norm(hh[3]) for hh in hist)
    for e, p, er, pr in hist:
        assert np.linalg.norm(e - er) / amp_e < 1e-10
        assert np.linalg.norm(p - pr) / amp_p < 1e-10
    assert rel_l2(hist[239][1], hist[239][3]) < 1e-10     # t = 3.75 T: phi_eta at its peak
    assert rel_l2(hist[255][0], hist[255][2]) < 1e-10     # t = 4 T: eta at its peak


SHAPE_SHAPES = [(3, 5, 3, 2, 6, True, False), (3, 5, 3, 2, 4, False, True), (3, 4, 3, 1, 8, True, True),
                (3, 7, 2, 2, 3, False, False), (3, 4, 3, 2, 5, True, True), (3, 3, 4, 1, 7, False, True),
                (3, 6, 2, 2, 2, True, False), (3, 9, 2, 1, 1, True, True)]


@pytest.mark.parametrize("shape", SHAPE_SHAPES, ids=ids)
@pytest.mark.parametrize("variant", list(range(12)))
def test_every_cta_shape_matches_oracle(fnpf, shape, variant):
    """Each elements-per-CTA shape of the operator kernels (the autotuner's
    candidates, including ragged last CTAs) gives the oracle's operator in
    FP64 and FP32, and the oracle's solution through the stored-metric
    p-multigrid solve."""
    c = Case(fnpf, *shape, opts=fnpf.default_opts(rtol=1e-13, precond=fnpf.FNPF_PMG, max_iter=5000))
    c.gm.set_shapes(variant, variant)
    v64, v32, c64, c32 = c.gm.get_shapes()
    assert (v64, v32) == (variant, variant) and c64 == c32 and c64 >= 1
    op = oop.Operator(c.om, c.eta, c.h)
    x = c.rng.standard_normal(c.om.N)
    y_ref = op.A @ x
    y = torch.empty(c.om.N, dtype=torch.float64, device=c.dev)
    c.gm.apply(c.t(c.eta), c.t(x), y)
    y32 = torch.empty(c.om.N, dtype=torch.float32, device=c.dev)
    c.gm.apply_f32(c.t(c.eta).float(), c.t(x).float(), y32)
    torch.cuda.synchronize()
    assert rel_max(y.cpu().numpy(), y_ref) < 1e-12
    assert rel_max(y32.double().cpu().numpy(), y_ref) < 2e-6
    phi_ref = osolve.laplace_solve(c.om, c.eta, c.h, c.phis)
    phi = torch.zeros(c.om.N, dtype=torch.float64, device=c.dev)
    info = c.gm.laplace_solve(c.t(c.eta), c.t(c.phis), phi)
    assert info["status"] == 0
    assert rel_l2(phi.cpu().numpy(), phi_ref) < 1e-10


def test_set_shapes_rejects_out_of_range(fnpf):
    c = Case(fnpf, *SHAPE_SHAPES[0])
    for bad in [(-1, 0), (0, 12), (12, 0)]:
        with pytest.raises(fnpf.FnpfError) as e:
            c.gm.set_shapes(*bad)
        assert e.value.status == fnpf.FNPF_EINVAL
    c2 = Case(fnpf, *SHAPES[0])
    with pytest.raises(fnpf.FnpfError):
        c2.gm.set_shapes(1, 0)
