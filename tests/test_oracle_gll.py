"""Pins of the oracle's GLL rule against closed forms and exactness properties
(the nodal GLL basis underlies the paper's P_p spaces, Sec. 3.1)."""
import math

import numpy as np
import pytest

from oracle import gll


def test_closed_form_nodes_and_weights():
    r2, r3, r4 = gll.Rule(2), gll.Rule(3), gll.Rule(4)
    assert np.allclose(r2.xi, [-1, 0, 1], atol=1e-15)
    assert np.allclose(r2.w, [1 / 3, 4 / 3, 1 / 3], atol=1e-15)
    s5 = 1 / math.sqrt(5)
    assert np.allclose(r3.xi, [-1, -s5, s5, 1], atol=1e-15)
    assert np.allclose(r3.w, [1 / 6, 5 / 6, 5 / 6, 1 / 6], atol=1e-15)
    s = math.sqrt(3 / 7)
    assert np.allclose(r4.xi, [-1, -s, 0, s, 1], atol=1e-15)
    assert np.allclose(r4.w, [1 / 10, 49 / 90, 32 / 45, 49 / 90, 1 / 10], atol=1e-15)


@pytest.mark.parametrize("p", range(1, 9))
def test_quadrature_exactness(p):
    r = gll.Rule(p)
    assert abs(r.w.sum() - 2) < 1e-14
    for m in range(0, 2 * p):              # exact up to degree 2p - 1
        exact = (1 - (-1) ** (m + 1)) / (m + 1)
        assert abs(r.w @ r.xi ** m - exact) < 1e-13
    m = 2 * p                              # not exact at degree 2p (Lobatto, not Gauss)
    assert abs(r.w @ r.xi ** m - 2 / (m + 1)) > 1e-6


@pytest.mark.parametrize("p", range(1, 9))
def test_derivative_matrix(p):
    r = gll.Rule(p)
    for m in range(0, p + 1):              # exact on polynomials of degree <= p
        d = r.D @ r.xi ** m
        ref = m * r.xi ** (m - 1) if m > 0 else 0 * r.xi
        assert np.max(np.abs(d - ref)) < 1e-12 * max(1, p * p)
    # closed form in terms of P_p at the nodes (Deville, Fischer & Mund 2002, Sec. 2.4)
    P, _ = gll.legendre(p, r.xi)
    Dc = np.zeros((p + 1, p + 1))
    for i in range(p + 1):
        for j in range(p + 1):
            if i != j:
                Dc[i, j] = P[i] / (P[j] * (r.xi[i] - r.xi[j]))
    Dc[0, 0], Dc[p, p] = -p * (p + 1) / 4, p * (p + 1) / 4
    assert np.max(np.abs(Dc - r.D)) < 1e-12 * p * p
    # antisymmetry about the centre, rows sum to zero
    assert np.max(np.abs(r.D + r.D[::-1, ::-1])) < 1e-12 * p * p
    assert np.max(np.abs(r.D.sum(axis=1))) < 1e-12 * p * p


def test_nodes_are_roots_of_legendre_derivative():
    for p in range(2, 9):
        r = gll.Rule(p)
        _, dP = gll.legendre(p, r.xi[1:-1])
        assert np.max(np.abs(dP)) < 1e-12
