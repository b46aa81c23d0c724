"""Tangent-linear model of the oracle's discrete RK4 step (test infrastructure
only): the exact directional derivative of the discrete map
(eta_n, phi_n, h) -> (eta_{n+1}, phi_{n+1}) by the complex-step method
(Squire & Trapp 1998; Martins, Sturdza & Alonso 2003): for an analytic map F,
F'(x) d = Im F(x + i eps d) / eps with no subtractive cancellation, so eps can
be tiny (1e-30) and the derivative is exact to rounding.  The oracle's
arithmetic is analytic in (eta, phi, h) -- |det J| is written as
det J sign(Re det J) -- so the same code serves.  Parity of the GPU adjoint
with this TLM is the dot-product identity <lam, J d> = <J^T lam, d>.
"""
import numpy as np

from . import surface

EPS = 1e-30


def step_tlm(mesh, h, eta, phis, dt, g, d_eta, d_phis, d_h=None, relax=None, t=0.0):
    """(d eta_{n+1}, d phi_{n+1}) for the perturbation (d_eta, d_phis, d_h)
    of one RK4 step (with the relaxation step of Sec. 3.3 when relax =
    (cr, gen, wave) is given)."""
    e = eta + 1j * EPS * d_eta
    p = phis + 1j * EPS * d_phis
    hh = h + 1j * EPS * (d_h if d_h is not None else 0.0)
    if relax is None:
        eo, po = surface.rk4_step(mesh, hh, e, p, dt, g)
    else:
        cr, gen, wave = relax
        eo, po = surface.relaxation_step(mesh, hh, e, p, t, dt, g, cr, gen, wave)
    return np.imag(eo) / EPS, np.imag(po) / EPS
