"""Over-integrated free-surface right-hand side (fnpf_set_dealias; paper Sec.
3.2) against the oracle's oracle/dealias.py: the right-hand side alone and
RK4 steps (host-driven and graph-replayed), 2D and 3D, box and curved
isoparametric meshes, walls and periodic."""
import numpy as np
import pytest
import torch

from oracle import dealias as odl
from oracle import solve as osolve
from paper_2506_09435_gb300 import workloads as W
from tests.pairs import Case, rel_l2, rel_max

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("shape,M", [((3, 4, 3, 2, 4, True, False), 8), ((3, 3, 3, 2, 6, False, False), 13),
                                     ((2, 6, 1, 2, 5, True, False), 9), ((3, 3, 2, 1, 3, True, True), 4)],
                         ids=["3d_PW_p4_M8", "3d_WW_p6_M13", "2d_p5_M9", "3d_PP_p3_M4"])
def test_dealiased_rhs_matches_oracle(fnpf, shape, M):
    c = Case(fnpf, *shape, amp=0.08, hvar=0.1)
    w = c.rng.standard_normal(c.om.ns) * 0.1
    c.gm.set_dealias(M)
    de, dp = (torch.empty(c.om.ns, dtype=torch.float64, device=c.dev) for _ in range(2))
    c.gm.zakharov_rhs(c.t(c.eta), c.t(c.phis), c.t(w), de, dp)
    torch.cuda.synchronize()
    re, rp = odl.zakharov_rhs_dealiased(c.om, c.eta, c.phis, w, 9.81, M)
    assert rel_max(de.cpu().numpy(), re) < 1e-12
    assert rel_max(dp.cpu().numpy(), rp) < 1e-12


def test_dealiased_rhs_on_curved_ogrid_matches_oracle(fnpf):
    """Isoparametric annulus (the cylinder O-grid map, reduced): the Gauss-point
    metric comes from the interpolated node coordinates on both sides."""
    from oracle import mesh as omesh
    nth, nr, p = 8, 3, 4
    box = omesh.Mesh(3, nth, nr, 1, p, periodic_x=True, periodic_y=False, Lx=2 * np.pi, Ly=1.0)
    th, sr = box.surface_coords()
    X, Y = W.ogrid_map(th, sr, a=1.0, R=4.0)
    om = omesh.Mesh(3, nth, nr, 1, p, periodic_x=True, periodic_y=False, X=X, Y=Y)
    h = np.full(om.ns, 1.0)
    gm = fnpf.Mesh(3, nth, nr, 1, p, True, False, h, X=X, Y=Y)
    rng = np.random.default_rng(4)
    eta = 0.05 * np.cos(X) * np.sin(0.5 * Y)
    phis = 0.1 * np.sin(X + 0.3 * Y)
    w = 0.1 * rng.standard_normal(om.ns)
    gm.set_dealias(9)
    dev = torch.device("cuda:0")
    t = lambda a: torch.tensor(a, dtype=torch.float64, device=dev)
    de, dp = torch.empty(om.ns, dtype=torch.float64, device=dev), torch.empty(om.ns, dtype=torch.float64, device=dev)
    gm.zakharov_rhs(t(eta), t(phis), t(w), de, dp)
    torch.cuda.synchronize()
    re, rp = odl.zakharov_rhs_dealiased(om, eta, phis, w, 9.81, 9)
    assert rel_max(de.cpu().numpy(), re) < 1e-12
    assert rel_max(dp.cpu().numpy(), rp) < 1e-12


@pytest.mark.parametrize("shape,M", [((3, 4, 3, 2, 4, True, True), 8), ((2, 6, 1, 2, 5, True, False), 9)],
                         ids=["3d_p4", "2d_p5"])
def test_dealiased_rk4_steps_match_oracle(fnpf, shape, M):
    """Three RK4 steps (the second and third replay the captured step graph)."""
    opts = fnpf.default_opts(rtol=1e-13, precond=fnpf.FNPF_PMG, max_iter=50000)
    c = Case(fnpf, *shape, amp=0.08, opts=opts)
    c.gm.set_dealias(M)
    eta, phis = c.t(c.eta), c.t(c.phis)
    e_r, p_r = c.eta, c.phis
    dt = 0.02
    for k in range(3):
        c.gm.rk4_step(eta, phis, k * dt, dt)
        e_r, p_r = odl.rk4_step_dealiased(c.om, c.h, e_r, p_r, dt, 9.81, M)
    torch.cuda.synchronize()
    assert rel_l2(eta.cpu().numpy(), e_r) < 1e-10
    assert rel_l2(phis.cpu().numpy(), p_r) < 1e-10


def test_set_dealias_validates_and_blocks_the_adjoint(fnpf):
    c = Case(fnpf, 3, 3, 3, 1, 4, True, True)
    for bad in (3, 4, 18, -1):
        with pytest.raises(fnpf.FnpfError) as e:
            c.gm.set_dealias(bad)
        assert e.value.status == fnpf.FNPF_EINVAL
    c.gm.set_dealias(7)
    z = c.t(np.zeros(c.om.ns))
    with pytest.raises(fnpf.FnpfError) as e:
        c.gm.step_adjoint(c.t(c.eta), c.t(c.phis), z, z, z.clone(), z.clone())
    assert e.value.status == fnpf.FNPF_EUNSUPPORTED
    c.gm.set_dealias(0)
