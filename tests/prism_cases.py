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


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))
