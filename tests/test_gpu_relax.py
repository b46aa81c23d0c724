"""Relaxation zones (Sec. 3.3, Step 4.7): generation of a linear incident
wave (ramped in over five periods) and absorption, applied after each RK4
step; parity with the oracle on a short flume over the bar bathymetry, and the
mixed-precision form against the FP64 path."""
import numpy as np
import pytest
import torch

from oracle import mesh as omesh
from oracle import surface as osurf
from paper_2506_09435_gb300 import workloads as W
from tests.pairs import rel_l2

pytestmark = pytest.mark.gpu


def flume(fnpf, nx, ny, nz, p, Lx, opts):
    d = W.bar_flume(nx=nx, ny=ny, nz=nz, p=p, Lx=Lx)
    d["zone"] = Lx / 4
    om = omesh.Mesh(3, nx, ny, nz, p, periodic_x=False, periodic_y=False, Lx=Lx, Ly=d["Ly"])
    x, y = om.surface_coords()
    h = W.bar_depth(x * 38.0 / Lx)          # the bar shape squeezed into the short flume
    gm = fnpf.Mesh(3, nx, ny, nz, p, False, False, h, Lx=Lx, Ly=d["Ly"], g=d["g"], opts=opts)
    cr, gen = W.flume_zones(d, x)
    wave = W.flume_wave(d)
    gm.set_relaxation(cr, gen, **wave)
    return d, om, gm, x, h, cr, gen, wave


def test_relaxed_steps_match_oracle(fnpf):
    d, om, gm, x, h, cr, gen, wave = flume(fnpf, 12, 2, 2, 3, 12.0, fnpf.default_opts(rtol=1e-13))
    dt = d["T"] / 100
    dev = torch.device("cuda:0")
    eta_r = np.zeros(om.ns)
    phi_r = np.zeros(om.ns)
    eta = torch.zeros(om.ns, dtype=torch.float64, device=dev)
    phis = torch.zeros_like(eta)
    for n in range(6):
        eta_r, phi_r = osurf.relaxation_step(om, h, eta_r, phi_r, n * dt, dt, d["g"], cr, gen, wave)
        gm.rk4_step(eta, phis, n * dt, dt)
    torch.cuda.synchronize()
    assert np.max(np.abs(eta_r)) > 0          # the generation zone has started the wave
    assert rel_l2(eta.cpu().numpy(), eta_r) < 1e-10
    assert rel_l2(phis.cpu().numpy(), phi_r) < 1e-10


def test_mixed_flume_matches_fp64_path(fnpf):
    """Mixed precision (FP32 operator and p-multigrid, FP64 defect correction) on
    a bar flume: the surface elevation after 40 steps agrees with the FP64 path
    to 1e-8 relative."""
    out = []
    for prec in (fnpf.FNPF_FP64, fnpf.FNPF_MIXED):
        o = fnpf.default_opts(rtol=1e-10, precision=prec, precond=fnpf.FNPF_PMG)
        d, om, gm, x, h, cr, gen, wave = flume(fnpf, 48, 4, 3, 4, 19.0, o)
        dt = d["T"] / 100
        eta = torch.zeros(om.ns, dtype=torch.float64, device=torch.device("cuda:0"))
        phis = torch.zeros_like(eta)
        for n in range(40):
            gm.rk4_step(eta, phis, n * dt, dt)
        torch.cuda.synchronize()
        out.append((eta.cpu().numpy(), phis.cpu().numpy()))
    assert np.max(np.abs(out[0][0])) > 1e-4
    assert rel_l2(out[1][0], out[0][0]) < 1e-8
    assert rel_l2(out[1][1], out[0][1]) < 1e-8
