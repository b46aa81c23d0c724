"""Linear potential flow (model FNPF_LINEAR; the paper's LPF, Sec. 1 and 2):
the Laplace problem on the still-water domain and the linear surface
conditions d eta/dt = w, d phi/dt = -g eta.  The GPU steps match the
oracle's linear RK4 (whose stability polynomial and dispersion relation are
pinned in test_oracle_time.py); the solver set-up done for the fixed geometry
at the first solve is reused by later ones."""
import numpy as np
import pytest
import torch

from oracle import solve as osolve
from oracle import surface as osurf
from paper_2506_09435_gb300 import workloads
from tests.pairs import Case, rel_l2, rel_max
from tests.test_gpu_parity import SHAPES, ids

pytestmark = pytest.mark.gpu


def lpf(fnpf, **kw):
    kw.setdefault("rtol", 1e-13)
    kw.setdefault("max_iter", 50000)
    return fnpf.default_opts(model=fnpf.FNPF_LINEAR, **kw)


@pytest.mark.parametrize("shape", [SHAPES[0], SHAPES[2], SHAPES[4], SHAPES[9]], ids=ids)
@pytest.mark.parametrize("precond,precision", [("jacobi", "fp64"), ("pmg", "fp64"), ("pmg", "mixed")])
def test_lpf_rk4_steps_match_oracle(fnpf, shape, precond, precision):
    """Four steps (the first host-driven, the rest replayed as step graphs
    that skip the kept set-up) against the oracle's linear RK4."""
    opts = lpf(fnpf, precond=fnpf.FNPF_PMG if precond == "pmg" else fnpf.FNPF_JACOBI,
               precision=fnpf.FNPF_MIXED if precision == "mixed" else fnpf.FNPF_FP64, inner_rtol=1e-5)
    c = Case(fnpf, *shape, opts=opts)
    dt = 0.01
    eta_r, phi_r = c.eta.copy(), c.phis.copy()
    eta, phis = c.t(c.eta), c.t(c.phis)
    for n in range(4):
        eta_r, phi_r = osurf.rk4_step(c.om, c.h, eta_r, phi_r, dt, 9.81, linear=True)
        c.gm.rk4_step(eta, phis, n * dt, dt)
    torch.cuda.synchronize()
    assert rel_l2(eta.cpu().numpy(), eta_r) < 1e-10
    assert rel_l2(phis.cpu().numpy(), phi_r) < 1e-10


def test_lpf_right_hand_side_is_linear(fnpf):
    c = Case(fnpf, *SHAPES[3], opts=lpf(fnpf))
    w = c.rng.standard_normal(c.om.ns)
    de = torch.empty(c.om.ns, dtype=torch.float64, device=c.dev)
    dp = torch.empty_like(de)
    c.gm.zakharov_rhs(c.t(c.eta), c.t(c.phis), c.t(w), de, dp)
    torch.cuda.synchronize()
    assert np.array_equal(de.cpu().numpy(), w)
    assert rel_max(dp.cpu().numpy(), -9.81 * c.eta) < 1e-15


@pytest.mark.parametrize("precond", ["jacobi", "pmg"])
def test_lpf_solve_uses_still_water_geometry_and_keeps_set_up(fnpf, precond):
    """An LPF solve with eta != 0 is the nonlinear solve on eta = 0; a second
    LPF solve with another eta (kept set-up) returns the same potential; and
    the oracle's solve on the flat geometry agrees."""
    pre = fnpf.FNPF_PMG if precond == "pmg" else fnpf.FNPF_JACOBI
    shape = SHAPES[3]
    cl = Case(fnpf, *shape, opts=lpf(fnpf, precond=pre))
    cn = Case(fnpf, *shape, opts=fnpf.default_opts(rtol=1e-13, precond=pre, max_iter=50000))
    zero = np.zeros(cl.om.ns)
    out = []
    for case, eta in ((cl, cl.eta), (cl, 0.5 * cl.eta), (cn, zero)):
        phi = torch.zeros(cl.om.N, dtype=torch.float64, device=cl.dev)
        assert case.gm.laplace_solve(case.t(eta), case.t(cl.phis), phi)["status"] == 0
        out.append(phi.cpu().numpy())
    assert rel_l2(out[0], out[2]) < 1e-13
    assert rel_l2(out[1], out[2]) < 1e-13
    phi_ref = osolve.laplace_solve(cl.om, zero, cl.h, cl.phis)
    assert rel_l2(out[0], phi_ref) < 1e-10


def test_lpf_standing_wave_2d_full_run_matches_oracle(fnpf):
    """The 2D 8 x 2, p = 4 standing-wave tank for 4 periods (256 RK4 steps,
    dt = T/64) in linear potential flow, against the oracle's linear steps:
    eta and phi_eta to 1e-10 relative to their amplitude over the run."""
    d = workloads.standing_wave_2d()
    c = Case(fnpf, 2, d["nx"], 1, d["nz"], d["p"], True, False, Lx=d["Lx"], h0=d["h0"], hvar=0.0,
             opts=lpf(fnpf, rtol=1e-12))
    h = np.full(c.om.ns, d["h0"])
    eta0, phi0 = workloads.standing_wave_state(d, c.x)
    T = workloads.period(d["k"], d["h0"], d["g"])
    dt = T / 64
    eta_r, phi_r = eta0.copy(), phi0.copy()
    eta, phis = c.t(eta0), c.t(phi0)
    err_e = err_p = amp_e = amp_p = 0.0
    for n in range(256):
        eta_r, phi_r = osurf.rk4_step(c.om, h, eta_r, phi_r, dt, d["g"], linear=True)
        c.gm.rk4_step(eta, phis, n * dt, dt)
        e, p = eta.cpu().numpy(), phis.cpu().numpy()
        err_e, err_p = max(err_e, np.linalg.norm(e - eta_r)), max(err_p, np.linalg.norm(p - phi_r))
        amp_e, amp_p = max(amp_e, np.linalg.norm(eta_r)), max(amp_p, np.linalg.norm(phi_r))
    assert err_e / amp_e < 1e-10 and err_p / amp_p < 1e-10


def test_lpf_adjoint_is_unsupported_and_model_is_validated(fnpf):
    c = Case(fnpf, *SHAPES[2], opts=lpf(fnpf))
    z = torch.zeros(c.om.ns, dtype=torch.float64, device=c.dev)
    with pytest.raises(fnpf.FnpfError) as e:
        c.gm.step_adjoint(c.t(c.eta), c.t(c.phis), z, z, z.clone(), z.clone(), None, 0.0, 0.01)
    assert e.value.status == fnpf.FNPF_EUNSUPPORTED
    with pytest.raises(fnpf.FnpfError) as e:
        c.gm.set_opts(fnpf.default_opts(model=7))
    assert e.value.status == fnpf.FNPF_EINVAL
