"""Pins of the oracle's over-integration of the nonlinear free-surface terms
(oracle/dealias.py; paper Sec. 3.2): the Gauss-point projection against exact
Legendre arithmetic (numpy.polynomial.legendre, independent of the oracle's
GLL code), reproduction of polynomial right-hand sides, and the dealiased
value of a squared top mode."""
import numpy as np
import numpy.polynomial.legendre as npl
import pytest

from oracle import dealias, gll
from oracle import mesh as omesh
from oracle import surface


def _poly_at(coef_leg, x):
    return npl.legval(x, coef_leg)


@pytest.mark.parametrize("p", [1, 2, 4, 6, 8])
def test_projection_reproduces_degree_p_polynomials(p):
    rng = np.random.default_rng(p)
    xi = gll.nodes(p)[0]
    for M in (p + 1, (3 * (p + 1) + 1) // 2, 2 * p + 1):
        xq, _ = dealias.gauss_rule(M)
        c = rng.standard_normal(p + 1)
        got = dealias.projection_matrix(p, M) @ _poly_at(c, xq)
        assert np.max(np.abs(got - _poly_at(c, xi))) < 1e-12 * np.max(np.abs(c)) * (p + 1)


@pytest.mark.parametrize("p,M", [(3, 6), (4, 7), (6, 13), (8, 12)])
def test_projection_is_the_truncated_legendre_series(p, M):
    """For f of degree d <= 2M - 1 - p the Gauss sums are exact: the result is
    the Legendre series of f truncated after degree p, at the GLL nodes."""
    rng = np.random.default_rng(10 * p + M)
    d = 2 * M - 1 - p
    c = rng.standard_normal(d + 1)
    xq, _ = dealias.gauss_rule(M)
    got = dealias.projection_matrix(p, M) @ _poly_at(c, xq)
    want = _poly_at(c[:p + 1], gll.nodes(p)[0])
    assert np.max(np.abs(got - want)) < 1e-12 * np.max(np.abs(c)) * d


def test_squared_top_mode_loses_its_aliased_part():
    """One 2D element (walls), eta = phi = 0 and w = P_p(r) at the nodes:
    d eta/dt = w exactly, d phi/dt = 1/2 Pi(P_p^2), the truncated Legendre
    series of P_p^2 (which collocation would fold onto the nodes)."""
    p, g = 5, 9.81
    m = omesh.Mesh(2, 1, 1, 1, p, periodic_x=False, Lx=2.0)
    x, _ = m.surface_coords()
    r = x - 1.0                                   # reference coordinate of the single element
    top = np.zeros(p + 1)
    top[p] = 1.0
    w = _poly_at(top, r)
    zero = np.zeros(m.ns)
    de, dp = dealias.zakharov_rhs_dealiased(m, zero, zero, w, g, M=2 * p + 1)
    sq = npl.legmul(top, top)                      # P_p^2, degree 2p
    want = 0.5 * _poly_at(sq[:p + 1], r)
    assert np.max(np.abs(de - w)) < 1e-13
    assert np.max(np.abs(dp - want)) < 1e-13
    assert np.max(np.abs(0.5 * w * w - want)) > 1e-2   # collocation differs here


@pytest.mark.parametrize("dim,p", [(3, 3), (3, 5), (2, 4)])
def test_low_degree_fields_give_the_collocation_rhs(dim, p):
    """On an affine walled box with eta, phi_eta and w linear in (x, y), both
    right-hand sides are polynomials of degree <= 2 <= p in each direction:
    the over-integrated right-hand side equals the collocation one."""
    m = omesh.Mesh(dim, 3, 2, 1, p, periodic_x=False, periodic_y=False, Lx=1.5, Ly=1.0)
    x, y = m.surface_coords()
    eta = 0.01 + 0.02 * x - 0.03 * y
    phis = 0.1 - 0.05 * x + 0.04 * y
    w = 0.2 + 0.1 * x + 0.07 * y
    ref = surface.zakharov_rhs(m, eta, phis, w, 9.81)
    for M in (p + 1, 2 * p + 1):
        got = dealias.zakharov_rhs_dealiased(m, eta, phis, w, 9.81, M)
        for a, b in zip(got, ref):
            assert np.max(np.abs(a - b)) < 1e-13 * max(1.0, np.max(np.abs(b)))
