"""Writes box_p6_8x8x2_trajectory.npz: the oracle's state of a reduced copy of
the 3D nonlinear periodic box (kh = 2, L = 1 m, Airy wave H/L = 0.05 plus the
seeded spectrum, seed 2, dt = T/100; 8 x 8 x 2 hexahedra of order p = 6, the
benchmark tank's element shape and order on a quarter of its columns) after 1
and after 20 classical RK4 steps (paper Sec. 3.2; Sec. 3.4 Steps 4.1-4.6).

Calls only the oracle and the seeded input generators; the Laplace solves are
Jacobi-preconditioned CG to ||r|| <= 1e-14 ||b||.  About 5 minutes on one core:

    python tests/golden/make_box_p6_trajectory.py
"""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import mesh, surface  # noqa: E402
from paper_2506_09435_gb300 import workloads as W  # noqa: E402

NXY, NZ, P, STEPS = 8, 2, 6, 20
OUT = os.path.join(HERE, "box_p6_8x8x2_trajectory.npz")


def initial_state():
    d = W.periodic_box_3d(nx=NXY, ny=NXY, nz=NZ, p=P, kh=2.0)
    m = mesh.Mesh(3, NXY, NXY, NZ, P, True, True, d["Lx"], d["Ly"])
    x, y = m.surface_coords()
    h = np.full(m.ns, d["h0"])
    eta, phis = W.airy_plus_spectrum_state(d, x, y, seed=2)
    dt = W.period(d["k"], d["h0"], d["g"]) / 100
    return d, m, h, eta, phis, dt


def main():
    d, m, h, eta, phis, dt = initial_state()
    out = dict(eta0=eta, phis0=phis, h=h, dt=dt)
    for n in range(STEPS):
        eta, phis = surface.rk4_step(m, h, eta, phis, dt, d["g"], method="pcg")
        if n == 0:
            out.update(eta1=eta, phis1=phis)
        print("step", n + 1, flush=True)
    out.update(eta20=eta, phis20=phis)
    np.savez_compressed(OUT, **out)
    print("wrote", OUT)


if __name__ == "__main__":
    main()
