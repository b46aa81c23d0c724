"""Pins of the oracle's cylinder-force functionals (oracle/wall.py): on a still
O-grid around a cylinder of radius a, with the volume potential of a given
smooth function sampled at the nodes, P = int n_x phi dS has the closed form
2 pi a J_1(kappa a) sinh(kappa h) / kappa for phi = cosh(kappa (z + h))
sin(kappa x), and K = int 1/2 |grad phi|^2 n_x dS equals an independent
fine-grid quadrature of the analytic gradient; both converge with the order."""
import math

import numpy as np
import pytest
from scipy import special

from oracle import mesh as omesh
from oracle import wall
from paper_2506_09435_gb300 import workloads as W


def ogrid(nth, nr, nz, p, a=1.0, R=3.0):
    box = omesh.Mesh(3, nth, nr, nz, p, periodic_x=True, periodic_y=False, Lx=2 * math.pi, Ly=1.0)
    th, s = box.surface_coords()
    X, Y = W.ogrid_map(th, s, a=a, R=R)
    return omesh.Mesh(3, nth, nr, nz, p, periodic_x=True, periodic_y=False, X=X, Y=Y), X, Y


def node_xyz(m, X, Y, h):
    """Physical coordinates of every volume node of the still mesh (eta = 0)."""
    ns, nv, p, nz = m.ns, m.nv, m.p, m.nz
    xi = m.rule.xi
    sig = np.array([(k // p + 0.5 * (1 + xi[k % p])) / nz if k < nv - 1 else 1.0 for k in range(nv)])
    z = (-h[None, :] + sig[:, None] * h[None, :]).ravel()
    return np.tile(X, nv), np.tile(Y, nv), z


def phi_fun(x, y, z, h, kap):
    return np.cosh(kap * (z + h)) * (np.sin(kap * x) + 0.3 * np.cos(kap * x) + 0.2 * y)


def grad2(x, y, z, h, kap):
    c, s = np.cosh(kap * (z + h)), np.sinh(kap * (z + h))
    f = np.sin(kap * x) + 0.3 * np.cos(kap * x) + 0.2 * y
    fx = kap * (np.cos(kap * x) - 0.3 * np.sin(kap * x))
    return (c * fx) ** 2 + (c * 0.2) ** 2 + (kap * s * f) ** 2


@pytest.mark.parametrize("p,tol_k", [(6, 1e-5), (8, 1e-7)])
def test_wall_functionals_converge_to_the_exact_integrals(p, tol_k):
    a, h0, kap = 1.0, 0.8, 1.3
    m, X, Y = ogrid(16, 4, 2, p, a=a)
    h = np.full(m.ns, h0)
    x, y, z = node_xyz(m, X, Y, h)
    phi = phi_fun(x, y, z, h0, kap)
    P, K = wall.wall_functionals(m, np.zeros(m.ns), h, phi, Mz=p + 2)
    # exact P: the y and cos terms integrate to zero against n_x = cos(theta) on the circle
    P_exact = 2 * math.pi * a * special.j1(kap * a) * math.sinh(kap * h0) / kap
    # K by a fine tensor Gauss rule in (theta, z) of the analytic gradient (n_x = cos theta)
    tq, tw = np.polynomial.legendre.leggauss(200)
    th = math.pi * (tq + 1)
    zq, zw = np.polynomial.legendre.leggauss(40)
    zz = 0.5 * h0 * (zq - 1)
    TH, ZZ = np.meshgrid(th, zz, indexing="ij")
    xw, yw = a * np.cos(TH), -a * np.sin(TH)
    K_exact = np.sum(np.outer(tw * math.pi, zw * 0.5 * h0) * 0.5 * grad2(xw, yw, ZZ, h0, kap) * np.cos(TH)) * a
    assert abs(P - P_exact) <= 1e-10 * abs(P_exact), (P, P_exact)
    assert abs(K - K_exact) <= tol_k * abs(K_exact), (K, K_exact)


def test_force_integral_is_linear_in_the_endpoint_potentials():
    """With one step between t_a and t_b the objective is
    P(y_b) - P(y_a) + dt/2 (K(y_a) + K(y_b)): checked against the functionals
    evaluated directly on the two states."""
    from oracle import solve, surface
    m, X, Y = ogrid(8, 2, 2, 3, a=1.0)
    h = np.full(m.ns, 1.0)
    eta = 0.01 * np.cos(X)
    phis = 0.05 * np.sin(X + 0.2)
    dt, g = 0.05, 9.81
    J = wall.force_integral(m, h, eta, phis, dt, g, 0, 1, Mz=5)
    e1, p1 = surface.rk4_step(m, h, eta, phis, dt, g)
    Pa, Ka = wall.wall_functionals(m, eta, h, solve.laplace_solve(m, eta, h, phis), 5)
    Pb, Kb = wall.wall_functionals(m, e1, h, solve.laplace_solve(m, e1, h, p1), 5)
    assert abs(J - (Pb - Pa + 0.5 * dt * (Ka + Kb))) <= 1e-14 * max(abs(Pa), abs(Pb))
