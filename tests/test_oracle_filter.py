"""Pins of the oracle's modal filter (Sec. 3.2): weights by their closed form,
low-degree polynomials unchanged, a single top Legendre mode scaled by
exactly sigma_p^2 (sigma_p in 1D), alpha = 0 the identity."""
import numpy as np
import pytest
from numpy.polynomial import legendre as npleg

from oracle import filter as ofilter
from oracle import mesh as omesh


def test_weights_closed_form():
    s = ofilter.weights(6, 36.0, 4, 2)
    assert np.all(s[:3] == 1.0)
    assert s[6] == pytest.approx(np.exp(-36.0), rel=1e-14)
    assert s[4] == pytest.approx(np.exp(-36.0 * 0.5 ** 4), rel=1e-14)
    assert np.all(np.diff(s) <= 0)


@pytest.mark.parametrize("dim,p,cutoff", [(3, 6, 3), (3, 4, 2), (2, 5, 3), (3, 8, 5)])
def test_polynomials_up_to_the_cutoff_are_unchanged(dim, p, cutoff):
    m = omesh.Mesh(dim, 3, 2, 1, p, periodic_x=False, periodic_y=False, Lx=1.5, Ly=0.8)
    x, y = m.surface_coords()
    rng = np.random.default_rng(3)
    f = np.zeros(m.ns)
    for a in range(cutoff + 1):
        for b in range(cutoff + 1 if dim == 3 else 1):
            f += rng.standard_normal() * x ** a * y ** b
    g = ofilter.filter_surface(m, f, 10.0, 2, cutoff)
    assert np.max(np.abs(g - f)) < 1e-12 * np.max(np.abs(f))


@pytest.mark.parametrize("dim,p", [(3, 6), (3, 3), (2, 4), (2, 7)])
def test_top_mode_is_scaled_by_sigma_p(dim, p):
    """Element (1, 1) carries P_p(r) P_p(s) (P_p(r) in 2D), zero elsewhere;
    its interior nodes come out scaled by sigma_p^2 (sigma_p)."""
    m = omesh.Mesh(dim, 3, 3, 1, p, periodic_x=False, periodic_y=False)
    alpha, order, cutoff = 5.0, 2, p - 2
    xi = m.rule.xi
    c = np.zeros(p + 1)
    c[p] = 1.0
    Pp = npleg.legval(xi, c)
    e = 1 * m.nx + 1 if dim == 3 else 1
    cols = m.ecol[e]
    f = np.zeros(m.ns)
    if dim == 3:
        f[cols] = np.outer(Pp, Pp)
        inner = cols[1:p, 1:p]
    else:
        f[cols[:, 0]] = Pp
        inner = cols[1:p, 0]
    sp = ofilter.weights(p, alpha, order, cutoff)[p]
    g = ofilter.filter_surface(m, f, alpha, order, cutoff)
    expect = f[inner] * (sp * sp if dim == 3 else sp)
    assert np.max(np.abs(g[inner] - expect)) < 1e-12


def test_alpha_zero_is_identity():
    m = omesh.Mesh(3, 4, 3, 1, 5)
    f = np.random.default_rng(0).standard_normal(m.ns)
    assert np.max(np.abs(ofilter.filter_surface(m, f, 0.0, 2, 1) - f)) < 1e-13
