"""Modal filter of free-surface fields (Sec. 3.2; applied in Step 4.7): the
GPU filter matches the oracle's element by element, and RK4 steps with the
filter (host-driven and replayed as step graphs) match the oracle's steps
followed by the oracle's filter of eta and phi."""
import numpy as np
import pytest
import torch

from oracle import filter as ofilter
from oracle import surface as osurf
from tests.pairs import Case, rel_l2, rel_max
from tests.test_gpu_parity import SHAPES, ids

pytestmark = pytest.mark.gpu

PARAMS = [(36.0, 8, 3), (2.0, 2, 0), (0.5, 1, 2)]


@pytest.mark.parametrize("shape", [SHAPES[0], SHAPES[1], SHAPES[2], SHAPES[3], SHAPES[4], SHAPES[9]], ids=ids)
@pytest.mark.parametrize("alpha,order,cutoff", PARAMS)
def test_filter_matches_oracle(fnpf, shape, alpha, order, cutoff):
    c = Case(fnpf, *shape)
    cutoff = min(cutoff, c.p - 1)
    c.gm.set_filter(alpha, order, cutoff)
    f = c.rng.standard_normal(c.om.ns)
    ref = ofilter.filter_surface(c.om, f, alpha, order, cutoff)
    g = c.t(f)
    c.gm.filter_apply(g)
    torch.cuda.synchronize()
    assert rel_max(g.cpu().numpy(), ref) < 1e-13


@pytest.mark.parametrize("shape", [SHAPES[0], SHAPES[2], SHAPES[3]], ids=ids)
def test_filtered_rk4_steps_match_oracle(fnpf, shape):
    alpha, order, cutoff = 6.0, 4, 1
    c = Case(fnpf, *shape, opts=fnpf.default_opts(rtol=1e-13, precond=fnpf.FNPF_PMG, max_iter=5000))
    c.gm.set_filter(alpha, order, cutoff)
    dt = 0.01
    eta_r, phi_r = c.eta.copy(), c.phis.copy()
    eta, phis = c.t(c.eta), c.t(c.phis)
    for n in range(4):
        eta_r, phi_r = osurf.rk4_step(c.om, c.h, eta_r, phi_r, dt, 9.81)
        eta_r = ofilter.filter_surface(c.om, eta_r, alpha, order, cutoff)
        phi_r = ofilter.filter_surface(c.om, phi_r, alpha, order, cutoff)
        c.gm.rk4_step(eta, phis, n * dt, dt)
    torch.cuda.synchronize()
    assert rel_l2(eta.cpu().numpy(), eta_r) < 1e-10
    assert rel_l2(phis.cpu().numpy(), phi_r) < 1e-10


def test_filter_off_and_errors(fnpf):
    c = Case(fnpf, *SHAPES[3])
    f = c.t(c.rng.standard_normal(c.om.ns))
    with pytest.raises(fnpf.FnpfError) as e:
        c.gm.filter_apply(f)                         # no filter set
    assert e.value.status == fnpf.FNPF_EINVAL
    for bad in [(-1.0, 2, 0), (1.0, 0, 0), (1.0, 2, c.p), (float("nan"), 2, 0)]:
        with pytest.raises(fnpf.FnpfError) as e:
            c.gm.set_filter(*bad)
        assert e.value.status == fnpf.FNPF_EINVAL
    c.gm.set_filter(3.0, 2, 1)
    z = torch.zeros(c.om.ns, dtype=torch.float64, device=c.dev)
    with pytest.raises(fnpf.FnpfError) as e:
        c.gm.step_adjoint(c.t(c.eta), c.t(c.phis), z, z, z.clone(), z.clone(), None, 0.0, 0.01)
    assert e.value.status == fnpf.FNPF_EUNSUPPORTED
    c.gm.set_filter(0.0)                             # off: steps are the unfiltered ones
    eta_r, phi_r = osurf.rk4_step(c.om, c.h, c.eta, c.phis, 0.01, 9.81)
    eta, phis = c.t(c.eta), c.t(c.phis)
    c.gm.rk4_step(eta, phis, 0.0, 0.01)
    torch.cuda.synchronize()
    assert rel_l2(eta.cpu().numpy(), eta_r) < 1e-9
