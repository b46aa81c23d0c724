"""Free-surface right-hand side, ERK4, relaxation and diagnostics (oracle, test
infrastructure only).

Zakharov conditions, paper Sec. 2, Eqs. (kinematic_free_surface_strong) and
(dynamic_free_surface_strong):
    d eta/dt  = -grad~eta . grad~phi_eta + w (1 + grad~eta . grad~eta)
    d phi_eta/dt = -g eta - 1/2 grad~phi_eta . grad~phi_eta + 1/2 w^2 (1 + grad~eta . grad~eta)
Weak forms, Sec. 3.1.1, Eq. (free_surface_weak): mass matrix times the time
derivative equals the integral of the right-hand side against each test
function.  Readings:
  * GLL quadrature at the nodes with the lumped (diagonal) GLL mass, so the
    nodal time derivative is sum_e W_e f_e / sum_e W_e, where f_e uses the
    element-local horizontal gradients and W_e = w_i w_j |det H|;
  * the sign of the 1/2 |grad~phi|^2 term follows the strong form (Bernoulli);
    the printed weak form F_d carries the opposite sign on that term, which
    contradicts the strong form it is derived from.
ERK4: Sec. 3.2 (classical four-stage scheme, constant step).
Relaxation: Sec. 3.3, f <- (1 - C_r) f + C_r f_true.
"""
import numpy as np

from .solve import dtn, horizontal_jacobian, lumped_mass, surface_cols, surface_weights


def surface_gradient(mesh, f):
    """Element-local horizontal gradient of the surface field f at every element
    surface node: (f_x, f_y) of shape (C, n, n) each in 3D, f_x (C, n) in 2D."""
    D = mesh.rule.D
    cols = surface_cols(mesh)
    ft = f[cols]
    if mesh.dim == 3:
        fr = np.einsum("ia,caj->cij", D, ft)
        fs = np.einsum("jb,cib->cij", D, ft)
        H = horizontal_jacobian(mesh)                       # [..., m, a] = d x_m / d r_a
        HT = np.swapaxes(H, -1, -2)
        g = np.linalg.solve(HT, np.stack([fr, fs], -1)[..., None])[..., 0]
        return g[..., 0], g[..., 1]
    fr = np.einsum("ia,ca->ci", D, ft)
    return fr / horizontal_jacobian(mesh), None


def zakharov_rhs(mesh, eta, phis, w, g):
    """(d eta/dt, d phi_eta/dt) at every surface column."""
    cols = surface_cols(mesh)
    ex, ey = surface_gradient(mesh, eta)
    px, py = surface_gradient(mesh, phis)
    if mesh.dim == 3:
        ge_gp = ex * px + ey * py
        ge2 = ex * ex + ey * ey
        gp2 = px * px + py * py
    else:
        ge_gp, ge2, gp2 = ex * px, ex * ex, px * px
    wl, el = w[cols], eta[cols]
    f_eta = -ge_gp + wl * (1 + ge2)
    f_phi = -g * el - 0.5 * gp2 + 0.5 * wl * wl * (1 + ge2)
    W = surface_weights(mesh)
    M = lumped_mass(mesh)
    d_eta = np.zeros(mesh.ns, dtype=f_eta.dtype)
    d_phi = np.zeros(mesh.ns, dtype=f_phi.dtype)
    np.add.at(d_eta, cols.ravel(), (W * f_eta).ravel())
    np.add.at(d_phi, cols.ravel(), (W * f_phi).ravel())
    return d_eta / M, d_phi / M


def linear_rhs(mesh, eta, phis, w, g):
    """Linearised conditions (LPF, surface held at z = 0): d eta/dt = w,
    d phi/dt = -g eta."""
    return w.copy(), -g * eta


def rhs(mesh, h, eta, phis, g, linear=False, method="direct"):
    geom_eta = np.zeros_like(eta) if linear else eta
    w, _ = dtn(mesh, geom_eta, h, phis, method=method)
    f = linear_rhs if linear else zakharov_rhs
    return f(mesh, eta, phis, w, g)


def rk4_step(mesh, h, eta, phis, dt, g, linear=False, method="direct"):
    """One classical RK4 step of the state (eta, phi_eta)."""
    def F(e, p):
        return rhs(mesh, h, e, p, g, linear=linear, method=method)
    k1 = F(eta, phis)
    k2 = F(eta + 0.5 * dt * k1[0], phis + 0.5 * dt * k1[1])
    k3 = F(eta + 0.5 * dt * k2[0], phis + 0.5 * dt * k2[1])
    k4 = F(eta + dt * k3[0], phis + dt * k3[1])
    eta_n = eta + dt / 6 * (k1[0] + 2 * k2[0] + 2 * k3[0] + k4[0])
    phi_n = phis + dt / 6 * (k1[1] + 2 * k2[1] + 2 * k3[1] + k4[1])
    return eta_n, phi_n


def relax(f, f_true, cr):
    """Relaxation-zone blend f <- (1 - C_r) f + C_r f_true (Sec. 3.3)."""
    return (1 - cr) * f + cr * f_true


def incident_wave(x, y, h, t, amp, kx, ky, omega, phase, g, ramp_time):
    """Linear incident wave of Sec. 3.3's generation zone at time t, multiplied by
    the generation ramp min(1, t / ramp_time) (the paper ramps generation over five
    wave periods; reading: a linear ramp applied to the target).  The potential
    is the linear one evaluated at the (ramped) target elevation."""
    r = min(1.0, t / ramp_time)
    th = kx * x + ky * y - omega * t + phase
    k = np.hypot(kx, ky)
    eta = r * amp * np.cos(th)
    phi = r * (g * amp / omega) * np.cosh(k * (eta + h)) / np.cosh(k * h) * np.sin(th)
    return eta, phi


def relaxation_step(mesh, h, eta, phis, t, dt, g, cr, gen, wave, linear=False, method="direct"):
    """One RK4 step followed by the relaxation-zone blend with targets at t + dt:
    the incident wave where gen = 1, zero where gen = 0 (Sec. 3.3, Step 4.7)."""
    eta, phis = rk4_step(mesh, h, eta, phis, dt, g, linear=linear, method=method)
    x, y = mesh.surface_coords()
    te, tp = incident_wave(x, y, h, t + dt, g=g, **wave)
    te = np.where(gen != 0, te, 0.0)
    tp = np.where(gen != 0, tp, 0.0)
    return relax(eta, te, cr), relax(phis, tp, cr)


def mass(mesh, eta):
    return float(lumped_mass(mesh) @ eta)


def energy(mesh, h, eta, phis, g, method="direct"):
    """E = 1/2 phi^T A phi + 1/2 g sum M eta^2 (unit density)."""
    from .operator import Operator
    from .solve import laplace_solve
    op = Operator(mesh, eta, h)
    phi = laplace_solve(mesh, eta, h, phis, op=op, method=method)
    return 0.5 * float(phi @ (op.A @ phi)) + 0.5 * g * float(lumped_mass(mesh) @ (eta * eta))
