"""Pins of the oracle's free-surface right-hand side and ERK4 (Sec. 2, Zakharov
conditions; Sec. 3.2 ERK4) against closed forms: the RK4 stability polynomial
on the linearised system, the linear dispersion relation omega^2 = g k tanh(kh)
(Sec. 3.3), and conservation of mass and energy."""
import math

import numpy as np
import pytest

from oracle import mesh, solve, surface
from paper_2506_09435_gb300 import workloads


def c1_setup(p=4):
    d = workloads.standing_wave_2d(p=p)
    m = mesh.Mesh(2, d["nx"], 1, d["nz"], d["p"], periodic_x=True, Lx=d["Lx"])
    x, _ = m.surface_coords()
    h = np.full(m.ns, d["h0"])
    eta0, phi0 = workloads.standing_wave_state(d, x)
    return d, m, x, h, eta0, phi0


def test_rk4_equals_stability_polynomial_on_linear_system():
    """LPF mode on the fixed mesh: y_{n+1} = P(dt L) y_n with
    P(z) = 1 + z + z^2/2 + z^3/6 + z^4/24, L = [[0, DtN], [-g I, 0]]."""
    d, m, x, h, eta0, phi0 = c1_setup()
    g = d["g"]
    ns = m.ns
    dtn = np.zeros((ns, ns))
    for j in range(ns):
        e = np.zeros(ns)
        e[j] = 1
        dtn[:, j] = solve.dtn(m, np.zeros(ns), h, e)[0]
    L = np.block([[np.zeros((ns, ns)), dtn], [-g * np.eye(ns), np.zeros((ns, ns))]])
    T = workloads.period(d["k"], d["h0"], g)
    dt = T / 64
    Z = dt * L
    P = np.eye(2 * ns) + Z + Z @ Z / 2 + Z @ Z @ Z / 6 + Z @ Z @ Z @ Z / 24
    y = np.concatenate([eta0, 0.3 * eta0 + 1e-5 * np.sin(2 * x)])
    eta, phis = y[:ns].copy(), y[ns:].copy()
    for _ in range(12):
        eta, phis = surface.rk4_step(m, h, eta, phis, dt, g, linear=True)
        y = P @ y
    assert np.max(np.abs(np.concatenate([eta, phis]) - y)) < 1e-12 * np.max(np.abs(y))


@pytest.mark.slow
def test_standing_wave_period_matches_dispersion_relation():
    """Small-amplitude standing wave on the 2D 8 x 2, p = 4 tank, dt = T/64,
    four periods: the period of eta(x = 0, t) equals 2 pi / sqrt(g k tanh kh)."""
    d, m, x, h, eta, phis = c1_setup()
    g = d["g"]
    T = workloads.period(d["k"], d["h0"], g)
    dt = T / 64
    hist = [eta[0]]
    mass0 = surface.mass(m, eta)
    for _ in range(256):
        eta, phis = surface.rk4_step(m, h, eta, phis, dt, g)
        hist.append(eta[0])
    hist = np.array(hist)
    t = dt * np.arange(len(hist))
    s = np.sign(hist)
    idx = np.nonzero(s[:-1] * s[1:] < 0)[0]
    tz = t[idx] - hist[idx] * dt / (hist[idx + 1] - hist[idx])
    Tnum = 2 * np.mean(np.diff(tz))
    assert abs(Tnum / T - 1) < 1e-4, (Tnum, T)
    a = 1e-4 * d["h0"]
    assert abs(surface.mass(m, eta) - mass0) < 1e-10 * a * d["Lx"]


def test_zakharov_rhs_reduces_to_linear_for_flat_state():
    """At eta = 0 the nonlinear right-hand side is (w, -1/2 |grad phi|^2 + 1/2 w^2)."""
    d, m, x, h, _, _ = c1_setup()
    phis = 1e-3 * np.sin(x)
    w = solve.dtn(m, 0 * x, h, phis)[0]
    de, dp = surface.zakharov_rhs(m, 0 * x, phis, w, d["g"])
    assert np.max(np.abs(de - w)) < 1e-15
    px, _ = surface.surface_gradient(m, phis)
    # px at element nodes; node value of 1/2 (w^2 - phi_x^2) averaged with the surface weights
    f = 0.5 * (w[surface.surface_cols(m)] ** 2 - px ** 2)
    W = surface.surface_weights(m)
    num = np.zeros(m.ns)
    np.add.at(num, surface.surface_cols(m).ravel(), (W * f).ravel())
    assert np.max(np.abs(dp - num / surface.lumped_mass(m))) < 1e-15


def test_surface_gradient_exact_on_polynomials_3d():
    m = mesh.Mesh(3, 3, 2, 1, 4, periodic_x=False, periodic_y=False, Lx=1.2, Ly=0.7)
    x, y = m.surface_coords()
    f = 1 + 2 * x - 3 * y + x * x * y - y ** 4
    fx, fy = surface.surface_gradient(m, f)
    cols = surface.surface_cols(m)
    X, Y = x[cols], y[cols]
    assert np.max(np.abs(fx - (2 + 2 * X * Y))) < 1e-12
    assert np.max(np.abs(fy - (-3 + X * X - 4 * Y ** 3))) < 1e-12


def test_energy_nearly_conserved_nonlinear_3d():
    d = workloads.periodic_box_3d(nx=3, ny=2, nz=1, p=4)
    m = mesh.Mesh(3, 3, 2, 1, 4, periodic_x=True, periodic_y=True, Lx=d["Lx"], Ly=d["Ly"])
    x, y = m.surface_coords()
    h = np.full(m.ns, d["h0"])
    eta, phis = workloads.airy_plus_spectrum_state(d, x, y, steepness=0.01)
    g = d["g"]
    T = workloads.period(d["k"], d["h0"], g)
    E0 = surface.energy(m, h, eta, phis, g)
    M0 = surface.mass(m, eta)
    for _ in range(8):
        eta, phis = surface.rk4_step(m, h, eta, phis, T / 32, g)
    E1 = surface.energy(m, h, eta, phis, g)
    assert abs(E1 / E0 - 1) < 1e-4
    assert abs(surface.mass(m, eta) - M0) < 1e-5 * np.max(np.abs(eta)) * d["Lx"] * d["Ly"]


def test_relaxation_blend_and_target():
    """Pins of the relaxation step: C_r = 1 replaces the state by the target,
    C_r = 0 leaves it; the generation target at the ramp's end is the linear
    Airy wave (eta = a cos(kx - wt), phi_eta = (g a / w) sin(...) at z = 0 for
    deep ramps); the weight function is 1 at the edge and 0 at the target side."""
    assert abs(workloads.relaxation_weight(0.0) - 1) < 1e-15
    assert abs(workloads.relaxation_weight(1.0)) < 1e-15
    xi = np.linspace(0, 1, 11)
    assert np.all(np.diff(workloads.relaxation_weight(xi)) < 0)
    f = np.array([1.0, 2.0, 3.0])
    ft = np.array([5.0, 5.0, 5.0])
    assert np.array_equal(surface.relax(f, ft, np.array([0.0, 1.0, 0.5])), np.array([1.0, 5.0, 4.0]))
    x = np.linspace(0, 3, 7)
    h = np.full_like(x, 0.4)
    g = 9.81
    k = workloads.wavenumber(2 * math.pi / 2.02, 0.4, g)
    om = 2 * math.pi / 2.02
    assert abs(om ** 2 - g * k * math.tanh(k * 0.4)) < 1e-12
    e, p = surface.incident_wave(x, 0 * x, h, 20.0, 1e-9, k, 0.0, om, 0.0, g, 10.0)
    th = k * x - om * 20.0
    assert np.max(np.abs(e - 1e-9 * np.cos(th))) < 1e-24
    assert np.max(np.abs(p - g * 1e-9 / om * np.sin(th))) < 1e-7 * g * 1e-9 / om
    e2, _ = surface.incident_wave(x, 0 * x, h, 5.0, 1e-3, k, 0.0, om, 0.0, g, 10.0)
    assert np.max(np.abs(e2 - 0.5e-3 * np.cos(k * x - om * 5.0))) < 1e-15


def test_bar_depth_profile():
    x = np.array([0.0, 14.0, 17.0, 20.0, 21.0, 22.0, 23.5, 25.0, 30.0])
    assert np.allclose(workloads.bar_depth(x), [0.4, 0.4, 0.25, 0.1, 0.1, 0.1, 0.25, 0.4, 0.4])
    d = workloads.bar_flume()
    assert workloads.dof_counts(d) == (1660176, 103761)


def test_complex_step_tlm_matches_central_differences():
    """The oracle's tangent-linear model (complex step) against central finite
    differences of the real oracle, for perturbations of eta, phi and h."""
    from oracle import tlm
    m = mesh.Mesh(3, 3, 2, 2, 3, periodic_x=True, periodic_y=False)
    x, y = m.surface_coords()
    h = 0.4 + 0.05 * np.cos(2 * np.pi * x)
    eta = 0.02 * np.cos(2 * np.pi * x + 0.3) * (1 + 0.3 * y)
    phis = 0.05 * np.sin(2 * np.pi * x) + 0.01 * y
    rng = np.random.default_rng(3)
    de, dp, dh = (rng.standard_normal(m.ns) for _ in range(3))
    dt, g = 0.02, 9.81
    te, tp = tlm.step_tlm(m, h, eta, phis, dt, g, de, dp, dh)
    s = 1e-6
    ep, pp = surface.rk4_step(m, h + s * dh, eta + s * de, phis + s * dp, dt, g)
    em, pm = surface.rk4_step(m, h - s * dh, eta - s * de, phis - s * dp, dt, g)
    fe, fp = (ep - em) / (2 * s), (pp - pm) / (2 * s)
    assert np.linalg.norm(te - fe) / np.linalg.norm(fe) < 1e-6
    assert np.linalg.norm(tp - fp) / np.linalg.norm(fp) < 1e-6
    # and the real part of the complex evaluation is the plain step
    e0, p0 = surface.rk4_step(m, h, eta, phis, dt, g)
    ec, pc = surface.rk4_step(m, h + 0j, eta + 1e-30j * de, phis + 0j, dt, g)
    assert np.max(np.abs(ec.real - e0)) < 1e-15 and np.max(np.abs(pc.real - p0)) < 1e-15
