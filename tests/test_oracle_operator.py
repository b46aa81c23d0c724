"""Pins of the oracle's stiffness operator (weak Laplace form, Sec. 3.1.1,
Eq. Laplace_weak) and mesh numbering (Sec. 3.1.2, DOF tables of Sec. 4.1)."""
import math
import os

import numpy as np
import pytest
from numpy.polynomial import Polynomial

from oracle import gll, mesh, operator
from paper_2506_09435_gb300 import workloads
from tests.oracle_helpers import global_node_coords

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "dof_counts.txt")


def read_dof_table():
    rows = []
    for line in open(GOLDEN):
        if line.startswith("#") or not line.strip():
            continue
        f = line.split()
        rows.append(tuple(int(v) for v in f[:6]) + (" ".join(f[6:]),))
    return rows


@pytest.mark.parametrize("row", read_dof_table(), ids=lambda r: r[6][:40])
def test_dof_counts_match_paper_tables(row):
    nx, ny, nz, p, nvol, nsurf, _src = row
    m = mesh.Mesh(3, nx, ny, nz, p, periodic_x=True, periodic_y=True)
    assert m.N == nvol
    if nsurf >= 0:
        assert m.ns == nsurf
    d = dict(dim=3, nx=nx, ny=ny, nz=nz, p=p, periodic_x=True, periodic_y=True)
    assert workloads.dof_counts(d) == (m.N, m.ns)


def exact_1d_stiffness(p):
    """K_ab = int_{-1}^{1} l_a' l_b' dx, by exact polynomial integration of the
    cardinal polynomials built from their roots (independent of the D matrix)."""
    xi = gll.Rule(p).xi
    L = []
    for a in range(p + 1):
        others = [xi[m] for m in range(p + 1) if m != a]
        poly = Polynomial.fromroots(others)
        L.append((poly / poly(xi[a])).deriv())
    K = np.zeros((p + 1, p + 1))
    for a in range(p + 1):
        for b in range(p + 1):
            P = (L[a] * L[b]).integ()
            K[a, b] = P(1.0) - P(-1.0)
    return K


@pytest.mark.parametrize("p", [1, 2, 3, 5, 8])
def test_affine_element_matches_kronecker_form_3d(p):
    Lx, Ly, nx, ny, nz, h0, c = 0.9, 1.3, 3, 2, 2, 0.7, 0.05
    m = mesh.Mesh(3, nx, ny, nz, p, periodic_x=True, periodic_y=False, Lx=Lx, Ly=Ly)
    op = operator.Operator(m, np.full(m.ns, c), np.full(m.ns, h0))
    K = exact_1d_stiffness(p)
    W = np.diag(gll.Rule(p).w)
    dx, dy, dz = Lx / nx, Ly / ny, (h0 + c) / nz
    kron = lambda a, b, cc: np.kron(np.kron(a, b), cc)
    ref = (dy * dz / (2 * dx)) * kron(K, W, W) + (dx * dz / (2 * dy)) * kron(W, K, W) \
        + (dx * dy / (2 * dz)) * kron(W, W, K)
    for e in [0, m.E - 1, m.E // 2]:
        Ae = op.element_matrix(e)
        assert np.max(np.abs(Ae - ref)) < 1e-12 * np.max(np.abs(ref))


@pytest.mark.parametrize("p", [1, 2, 4, 7])
def test_affine_element_matches_kronecker_form_2d(p):
    Lx, nx, nz, h0 = 2 * math.pi, 8, 2, 1.0
    m = mesh.Mesh(2, nx, 1, nz, p, periodic_x=True, Lx=Lx)
    op = operator.Operator(m, np.zeros(m.ns), np.full(m.ns, h0))
    K = exact_1d_stiffness(p)
    W = np.diag(gll.Rule(p).w)
    dx, dz = Lx / nx, h0 / nz
    ref = (dz / dx) * np.kron(K, W) + (dx / dz) * np.kron(W, K)
    for e in range(m.E):
        assert np.max(np.abs(op.element_matrix(e) - ref)) < 1e-12 * np.max(np.abs(ref))


def test_global_assembly_equals_element_scatter():
    m = mesh.Mesh(3, 2, 1, 2, 3, periodic_x=True, periodic_y=True)   # single element in y
    x, y = m.surface_coords()
    eta = 0.04 * np.cos(2 * np.pi * x) * np.sin(2 * np.pi * y)
    h = 0.5 + 0.1 * np.sin(2 * np.pi * x)
    op = operator.Operator(m, eta, h)
    A = np.zeros((m.N, m.N))
    for e in range(m.E):
        g = m.glob[e]
        A[np.ix_(g, g)] += 0  # placeholder to keep shapes obvious
        Ae = op.element_matrix(e)
        for a in range(len(g)):
            for b in range(len(g)):
                A[g[a], g[b]] += Ae[a, b]
    assert np.max(np.abs(op.A.toarray() - A)) < 1e-12 * np.max(np.abs(A))


@pytest.mark.parametrize("dim", [2, 3])
def test_symmetry_and_constant_nullspace_curved(dim):
    m = mesh.Mesh(dim, 3, 2, 2, 4, periodic_x=True, periodic_y=False)
    x, y = m.surface_coords()
    eta = 0.05 * np.cos(2 * np.pi * x + 0.3) * (1 + 0.5 * y)
    h = 0.4 + 0.1 * np.sin(2 * np.pi * x)
    op = operator.Operator(m, eta, h)
    A = op.A
    assert abs(A - A.T).max() < 1e-13 * abs(A).max()
    assert np.max(np.abs(A @ np.ones(m.N))) < 1e-12 * abs(A).max()
    v = np.random.default_rng(0).standard_normal(m.N)
    assert v @ (A @ v) > 0
    assert np.max(np.abs(op.apply(v) - A @ v)) < 1e-12 * np.max(np.abs(A @ v))


def exact_energy_2d(u, v, h, eta, L, nxq=512, nzq=40):
    """int_0^L int_{-h(x)}^{eta(x)} grad u . grad v dz dx: periodic trapezoid in
    x, Gauss-Legendre in z (both spectrally accurate for these smooth data)."""
    xq = np.arange(nxq) * L / nxq
    gz, gw = np.polynomial.legendre.leggauss(nzq)
    tot = 0.0
    for xv in xq:
        lo, hi = -h(xv), eta(xv)
        z = lo + (gz + 1) * (hi - lo) / 2
        ux, uz = u(xv, z)
        vx, vz = v(xv, z)
        tot += (hi - lo) / 2 * np.sum(gw * (ux * vx + uz * vz))
    return tot * L / nxq


def test_curved_operator_converges_to_exact_energy_2d():
    """a_GLL(I u, I v) -> int grad u . grad v over the eta/h-following domain,
    exponentially in p (pins the curved metric terms and the bathymetry terms)."""
    L, h0 = 1.0, 0.35
    k = 2 * np.pi / L
    hf = lambda x: h0 * (1 + 0.2 * np.sin(k * x))
    ef = lambda x: 0.04 * np.cos(k * x + 0.4)
    u = lambda x, z: (-k * np.sin(k * x + 0.2) * (1 + z + z * z), np.cos(k * x + 0.2) * (1 + 2 * z))
    v = lambda x, z: (2 * k * np.cos(2 * k * x) * np.cosh(z), np.sin(2 * k * x) * np.sinh(z))
    uf = lambda x, z: np.cos(k * x + 0.2) * (1 + z + z * z)
    vf = lambda x, z: np.sin(2 * k * x) * np.cosh(z)
    ref = exact_energy_2d(u, v, hf, ef, L)
    errs = []
    for p in [2, 4, 6, 8]:
        m = mesh.Mesh(2, 4, 1, 2, p, periodic_x=True, Lx=L)
        xs, _ = m.surface_coords()
        eta, h = ef(xs), hf(xs)
        op = operator.Operator(m, eta, h)
        X, _, Z = global_node_coords(m, eta, h)
        errs.append(abs(uf(X, Z) @ (op.A @ vf(X, Z)) - ref) / abs(ref))
    assert errs[-1] < 1e-7, errs
    for a, b in zip(errs, errs[1:]):
        assert b < a / 8, errs


def test_curved_operator_converges_to_exact_energy_3d():
    L, h0 = 1.0, 0.3
    k = 2 * np.pi / L
    hf = lambda x, y: h0 * (1 + 0.15 * np.sin(k * x) * np.cos(k * y))
    ef = lambda x, y: 0.03 * np.cos(k * x + 0.4) * np.sin(k * y + 0.1)
    uf = lambda x, y, z: np.cos(k * x + 0.2) * np.cos(k * y) * (1 + z + z * z)
    ug = lambda x, y, z: (-k * np.sin(k * x + 0.2) * np.cos(k * y) * (1 + z + z * z),
                          -k * np.cos(k * x + 0.2) * np.sin(k * y) * (1 + z + z * z),
                          np.cos(k * x + 0.2) * np.cos(k * y) * (1 + 2 * z))
    vf = lambda x, y, z: np.sin(k * (x + y)) * np.cosh(z)
    vg = lambda x, y, z: (k * np.cos(k * (x + y)) * np.cosh(z), k * np.cos(k * (x + y)) * np.cosh(z),
                          np.sin(k * (x + y)) * np.sinh(z))
    nq = 96
    xq = np.arange(nq) * L / nq
    X2, Y2 = np.meshgrid(xq, xq, indexing="ij")
    gz, gw = np.polynomial.legendre.leggauss(30)
    lo, hi = -hf(X2, Y2), ef(X2, Y2)
    Z3 = lo[..., None] + (gz + 1)[None, None, :] * (hi - lo)[..., None] / 2
    Xb, Yb = X2[..., None], Y2[..., None]
    gu, gv = ug(Xb, Yb, Z3), vg(Xb, Yb, Z3)
    integrand = sum(a * b for a, b in zip(gu, gv))
    ref = np.sum(((hi - lo) / 2)[..., None] * gw * integrand) * (L / nq) ** 2
    errs = []
    for p in [2, 4, 6]:
        m = mesh.Mesh(3, 3, 3, 2, p, periodic_x=True, periodic_y=True, Lx=L, Ly=L)
        xs, ys = m.surface_coords()
        eta, h = ef(xs, ys), hf(xs, ys)
        op = operator.Operator(m, eta, h)
        X, Y, Z = global_node_coords(m, eta, h)
        errs.append(abs(uf(X, Y, Z) @ (op.A @ vf(X, Y, Z)) - ref) / abs(ref))
    assert errs[-1] < 1e-4, errs
    for a, b in zip(errs, errs[1:]):
        assert b < a / 8, errs
