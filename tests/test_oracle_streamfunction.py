"""A steady nonlinear travelling wave (stream-function theory, the paper's
nonlinear initial condition, Sec. 3.3) as an exact solution of the FNPF
equations: the generator is pinned by its own residual and by third-order
Stokes theory; the oracle carries the wave for one period and returns it to
its initial shape with an error that falls with p (Sec. 4's spectral
convergence on nonlinear waves).  A flipped sign of the 1/2 |grad phi|^2 term
(reading R7) gives errors of 0.2 H and more instead of 1e-3 H."""
import math

import numpy as np
import pytest

from oracle import mesh as omesh
from oracle import surface as osurf
from paper_2506_09435_gb300 import workloads as W


@pytest.mark.parametrize("kh", [1.0, 2.0])
@pytest.mark.parametrize("steep", [0.002, 0.01, 0.03])
def test_stream_function_celerity_matches_third_order_stokes(kh, steep):
    k, d = kh, 1.0
    L = 2 * math.pi / k
    wave = W.StreamFunctionWave(d, L, steep * L, N=24)
    assert wave.residual < 1e-12
    sig = math.tanh(k * d)
    c0 = math.sqrt(9.81 / k * sig)
    ka = k * steep * L / 2
    c_stokes = c0 * (1 + ka ** 2 * (9 - 10 * sig ** 2 + 9 * sig ** 4) / (16 * sig ** 4))
    assert abs(wave.c - c_stokes) / c0 < 2 * ka ** 4 + 1e-12
    x = np.linspace(0.0, L, 41)
    assert wave.eta(0.0) - wave.eta(L / 2) == pytest.approx(steep * L, rel=1e-12)
    assert np.allclose(wave.eta(x, wave.period()), wave.eta(x), atol=1e-12)


def propagate_one_period(p, nx=4, nz=2, steep=0.05, nsteps=128):
    d, wave = W.stream_function_tank_2d(nx=nx, nz=nz, p=p, steepness=steep)
    m = omesh.Mesh(2, nx, 1, nz, p, periodic_x=True, periodic_y=False, Lx=d["Lx"])
    x, _ = m.surface_coords()
    h = np.full(m.ns, d["h0"])
    eta, phis = wave.eta(x), wave.phis(x)
    T = wave.period()
    dt = T / nsteps
    for _ in range(nsteps):
        eta, phis = osurf.rk4_step(m, h, eta, phis, dt, d["g"])
    e_eta = np.max(np.abs(eta - wave.eta(x, T))) / wave.H
    ref = wave.phis(x, T)
    e_phi = np.max(np.abs(phis - ref)) / np.max(np.abs(ref))
    return e_eta, e_phi


def test_oracle_carries_stream_function_wave_with_spectral_convergence():
    errs = {p: propagate_one_period(p) for p in (4, 6, 8)}
    assert errs[6][0] < errs[4][0] and errs[8][0] < errs[6][0]
    assert errs[6][1] < errs[4][1] and errs[8][1] < errs[6][1]
    assert errs[8][0] < 1e-3 and errs[8][1] < 2e-4
    assert errs[4][0] / errs[8][0] > 20 and errs[4][1] / errs[8][1] > 50
