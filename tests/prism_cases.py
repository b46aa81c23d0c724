"""Seeded inputs of the prism solve and step tests (CPU harness and GPU): a
jittered triangulation of a walled tank with a bottom bump, a curved free
surface and a smooth surface potential (input generation only).  Field values
are computed at the oracle's surface node coordinates; both sides receive the
same arrays."""
import numpy as np

from oracle import prism as P
from paper_2506_09435_gb300 import workloads as W

G = 9.81


def mesh(p, nz, nx=3, ny=2, Lx=1.3, Ly=1.0, seed=7):
    v, t = W.triangulated_box(nx, ny, Lx, Ly, seed=seed)
    return v, t, P.PrismMesh(P.TriMesh(v, t, p), nz)


def fields(pm, amp=0.02):
    x, y = pm.tm.xs, pm.tm.ys
    eta = amp * np.cos(2.0 * x) * np.sin(3.0 * y)
    h = 0.6 - 0.1 * np.exp(-((x - 0.6) ** 2 + (y - 0.5) ** 2) / 0.05)
    phis = 0.01 * np.cos(x) * np.cosh(0.3 * y)
    return eta, h, phis


def standing_wave(pm, Lx=1.3, amp=0.01):
    """The first sloshing mode of the walled tank (eta = A cos(pi x / Lx),
    phis = 0) plus a small seeded transverse perturbation, over the bumped
    bottom of `fields`."""
    x, y = pm.tm.xs, pm.tm.ys
    u = W.uniform01(3, 2)
    eta = amp * np.cos(np.pi * x / Lx) + 0.1 * amp * (u[0] - 0.5) * np.cos(np.pi * y)
    _, h, _ = fields(pm)
    return eta, h, np.zeros_like(eta)


def complex_step_vjp(pm, eta, h, phis, lam, eps=1e-30):
    """(dJ/deta, dJ/dphis, dJ/dh) of J = lam . phi(eta, h, phis) for the
    oracle's solve, one complex step per surface node and argument."""
    ge, gp, gh = np.zeros(pm.ns), np.zeros(pm.ns), np.zeros(pm.ns)
    for c in range(pm.ns):
        e = np.zeros(pm.ns)
        e[c] = 1.0
        ge[c] = lam @ P.laplace_solve(pm, eta + 1j * eps * e, h + 0j, phis + 0j).imag / eps
        gh[c] = lam @ P.laplace_solve(pm, eta + 0j, h + 1j * eps * e, phis + 0j).imag / eps
        gp[c] = lam @ P.laplace_solve(pm, eta + 0j, h + 0j, phis + 1j * eps * e).imag / eps
    return ge, gp, gh


def complex_step_step_vjp(pm, h, eta, phis, lam_e, lam_p, dt, linear=False, eps=1e-30):
    """J^T lam of one oracle RK4 step, entry by entry: one complex step per
    unit direction in eta, phis and h."""
    out = []
    for which in range(3):
        g = np.zeros(pm.ns)
        for c in range(pm.ns):
            d = [np.zeros(pm.ns) for _ in range(3)]
            d[which][c] = 1.0
            ce, cp = P.rk4_step(pm, h + 1j * eps * d[2], eta + 1j * eps * d[0], phis + 1j * eps * d[1], dt, G,
                                linear=linear)
            g[c] = lam_e @ (ce.imag / eps) + lam_p @ (cp.imag / eps)
        out.append(g)
    return out


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def flume(p, nz, nx=8, ny=2, Lx=4.0, Ly=0.5, h0=0.4, T=1.0, amp=0.005, seed=3):
    """A triangulated walled flume of depth h0 with a generation zone over
    [0, 1] and an absorption zone over [Lx - 1, Lx] (the relaxation weight and
    the linear incident wave of the structured flume workloads)."""
    v, t = W.triangulated_box(nx, ny, Lx, Ly, seed=seed)
    pm = P.PrismMesh(P.TriMesh(v, t, p), nz)
    omega = 2.0 * np.pi / T
    desc = dict(zone=1.0, Lx=Lx, amp=amp, k=W.wavenumber(omega, h0, G), omega=omega, T=T)
    cr, gen = W.flume_zones(desc, pm.tm.xs)
    return v, t, pm, np.full(pm.ns, h0), cr, gen, W.flume_wave(desc)
