"""The GPU path carries a steady nonlinear stream-function wave for one period
(one wavelength, 2D periodic tank, kh = 1, H/L = 0.05): it matches the
oracle's run and the exact travelling wave, with errors falling in p and h."""
import numpy as np
import pytest
import torch

from oracle import mesh as omesh
from oracle import surface as osurf
from paper_2506_09435_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def gpu_run(fnpf, p, nx, nz=2, steep=0.05, nsteps=128, precond=None):
    d, wave = W.stream_function_tank_2d(nx=nx, nz=nz, p=p, steepness=steep)
    pre = fnpf.FNPF_PMG if precond == "pmg" else fnpf.FNPF_JACOBI
    gm = fnpf.Mesh(2, nx, 1, nz, p, True, False, np.full(p * nx, d["h0"]), Lx=d["Lx"], g=d["g"],
                   opts=fnpf.default_opts(rtol=1e-13, max_iter=50000, precond=pre))
    x, _ = gm.surface_coords()
    dev = torch.device("cuda:0")
    eta = torch.tensor(wave.eta(x), dtype=torch.float64, device=dev)
    phis = torch.tensor(wave.phis(x), dtype=torch.float64, device=dev)
    T = wave.period()
    dt = T / nsteps
    for n in range(nsteps):
        gm.rk4_step(eta, phis, n * dt, dt)
    torch.cuda.synchronize()
    e, ph = eta.cpu().numpy(), phis.cpu().numpy()
    ref = wave.phis(x, T)
    return e, ph, (np.max(np.abs(e - wave.eta(x, T))) / wave.H, np.max(np.abs(ph - ref)) / np.max(np.abs(ref)))


def test_gpu_stream_function_period_matches_oracle_run(fnpf):
    p, nx = 6, 4
    e, ph, _ = gpu_run(fnpf, p, nx, precond="pmg")
    d, wave = W.stream_function_tank_2d(nx=nx, p=p)
    m = omesh.Mesh(2, nx, 1, 2, p, periodic_x=True, periodic_y=False, Lx=d["Lx"])
    x, _ = m.surface_coords()
    h = np.full(m.ns, d["h0"])
    eta, phis = wave.eta(x), wave.phis(x)
    dt = wave.period() / 128
    for _ in range(128):
        eta, phis = osurf.rk4_step(m, h, eta, phis, dt, d["g"])
    assert np.linalg.norm(e - eta) / np.linalg.norm(eta) < 1e-9
    assert np.linalg.norm(ph - phis) / np.linalg.norm(phis) < 1e-9


def test_gpu_stream_function_converges_in_p_and_h(fnpf):
    ep = {p: gpu_run(fnpf, p, 4)[2] for p in (3, 4, 5, 6, 7, 8)}
    for p in (4, 5, 6, 7, 8):
        assert ep[p][1] < ep[p - 1][1], ep
    assert ep[8][0] < 1e-3 and ep[8][1] < 2e-4
    # horizontal refinement at p = 4 (the vertical discretisation is held
    # fixed, so the rate is that of the horizontal error until it dominates)
    eh = {nx: gpu_run(fnpf, 4, nx)[2] for nx in (2, 4, 8)}
    assert eh[4][0] < eh[2][0] / 2.5 and eh[8][0] < eh[4][0] / 2.5, eh
    assert eh[4][1] < eh[2][1] / 4 and eh[8][1] < eh[4][1] / 4, eh
