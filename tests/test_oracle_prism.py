"""Pins of the prism oracle (oracle/prism.py): extruded prisms over an
unstructured triangular surface mesh (Sec. 3.1.2).

  * triangle nodes: count, vertices, edge nodes at the GLL points, symmetry;
  * triangle quadrature: exact integrals of barycentric monomials,
    int_T l1^a l2^b l3^c = 2 |T| a! b! c! / (a + b + c + 2)!;
  * nodal basis: cardinal at the nodes, reproduces every polynomial of degree
    <= p and its derivatives;
  * numbering: every shared node gets one position from all its triangles;
  * element matrix on a flat prism = the Kronecker form built from the
    triangle's stiffness and mass integrated exactly in closed form (monomial
    integrals, no quadrature) and the GLL vertical mass / exact 1D stiffness;
  * assembled operator: symmetric, constants in its null space, positive
    semi-definite on a curved (eta-following) mesh; a(I u, I v) converges to
    int grad u . grad v over a domain with a curved surface and a bottom bump
    (integrated independently in physical coordinates), which a wrong term
    of the vertical metric breaks;
  * Laplace solve + w: a constant potential is reproduced; the manufactured
    harmonic potential cosh(kappa (z + h)) cos(kx x) cos(ky y) gives the exact
    Dirichlet-to-Neumann map with errors falling exponentially in p and at
    rates approaching p under refinement (flat and curved eta)."""
import itertools
import math

import numpy as np
import pytest

from oracle import gll
from oracle import prism as P
from paper_2506_09435_gb300 import workloads as W


@pytest.mark.parametrize("p", [1, 2, 3, 4, 5])
def test_triangle_nodes(p):
    r, s = P.tri_nodes(p)
    assert len(r) == (p + 1) * (p + 2) // 2
    pts = set(zip(np.round(r, 12), np.round(s, 12)))
    assert {(-1.0, -1.0), (1.0, -1.0), (-1.0, 1.0)} <= pts
    xi = gll.nodes(p)[0]
    edge = np.sort(r[np.isclose(s, -1.0)])
    assert np.allclose(edge, xi, atol=1e-14)                  # edge A-B carries the GLL points
    assert np.allclose(np.sort(s[np.isclose(r, -1.0)]), xi, atol=1e-14)
    hyp = np.isclose(r + s, 0.0)
    assert hyp.sum() == p + 1
    assert pts == set(zip(np.round(s, 12), np.round(r, 12)))  # mirror r <-> s


@pytest.mark.parametrize("n", [2, 3, 4, 5, 6])
def test_triangle_quadrature_exact(n):
    r, s, w = P.tri_quadrature(n)
    lb, lc = (1 + r) / 2, (1 + s) / 2
    la = 1 - lb - lc
    for a, b, c in itertools.product(range(2 * n), repeat=3):
        if a + b + c > 2 * n - 2:
            continue
        exact = 2 * 2 * math.factorial(a) * math.factorial(b) * math.factorial(c) / math.factorial(a + b + c + 2)
        assert abs((w * la ** a * lb ** b * lc ** c).sum() - exact) < 1e-14
    assert abs(w.sum() - 2.0) < 1e-14


@pytest.mark.parametrize("p", [1, 2, 3, 4])
def test_nodal_basis(p):
    rn, sn = P.tri_nodes(p)
    L = P.tri_basis(p, rn, sn)[0]
    assert np.allclose(L, np.eye(len(rn)), atol=1e-12)
    rq, sq, _ = P.tri_quadrature(p + 2)
    L, Lr, Ls = P.tri_basis(p, rq, sq)
    for a, b in itertools.product(range(p + 1), repeat=2):
        if a + b > p:
            continue
        f = rn ** a * sn ** b
        assert np.allclose(L @ f, rq ** a * sq ** b, atol=1e-12)
        assert np.allclose(Lr @ f, a * rq ** max(a - 1, 0) * sq ** b if a else 0 * rq, atol=1e-11)
        assert np.allclose(Ls @ f, b * rq ** a * sq ** max(b - 1, 0) if b else 0 * rq, atol=1e-11)


@pytest.mark.parametrize("p", [1, 2, 3])
def test_numbering_is_conforming(p):
    v, t = W.triangulated_box(4, 3, 2.0, 1.0)
    tm = P.TriMesh(v, t, p)
    nedge = len({(min(a, b), max(a, b)) for tr in t for a, b in ((tr[0], tr[1]), (tr[1], tr[2]), (tr[0], tr[2]))})
    assert tm.ns == len(v) + nedge * (p - 1) + len(t) * (p - 1) * (p - 2) // 2
    rn, sn = P.tri_nodes(p)
    lb, lc = (1 + rn) / 2, (1 + sn) / 2
    for e, (A, B, C) in enumerate(t):
        X = (1 - lb - lc)[:, None] * v[A] + lb[:, None] * v[B] + lc[:, None] * v[C]
        assert np.allclose(X[:, 0], tm.xs[tm.nodes[e]], atol=1e-14)
        assert np.allclose(X[:, 1], tm.ys[tm.nodes[e]], atol=1e-14)
    assert len(np.unique(np.round(np.stack([tm.xs, tm.ys], 1), 12), axis=0)) == tm.ns


def exact_triangle_matrices(p, A, B, C):
    """Stiffness and mass of the order-p nodal basis on the affine triangle
    ABC, integrated exactly: the cardinal functions in monomials u^a v^b
    (u, v the barycentric coordinates of B and C), int_T u^a v^b dr ds =
    4 a! b! / (a + b + 2)!."""
    rn, sn = P.tri_nodes(p)
    ex = [(a, b) for b in range(p + 1) for a in range(p + 1 - b)]
    un, vn = (1 + rn) / 2, (1 + sn) / 2
    Cc = np.linalg.inv(np.array([[u ** a * vv ** b for a, b in ex] for u, vv in zip(un, vn)]))

    def I(a, b):
        return 0.0 if a < 0 or b < 0 else 4.0 * math.factorial(a) * math.factorial(b) / math.factorial(a + b + 2)

    m = len(ex)
    Mm, Srr, Srs, Sss = (np.zeros((m, m)) for _ in range(4))
    for i, (a1, b1) in enumerate(ex):
        for j, (a2, b2) in enumerate(ex):
            Mm[i, j] = I(a1 + a2, b1 + b2)
            Srr[i, j] = a1 * a2 / 4.0 * I(a1 + a2 - 2, b1 + b2)
            Srs[i, j] = a1 * b2 / 4.0 * I(a1 + a2 - 1, b1 + b2 - 1)
            Sss[i, j] = b1 * b2 / 4.0 * I(a1 + a2, b1 + b2 - 2)
    J2 = np.array([[B[0] - A[0], C[0] - A[0]], [B[1] - A[1], C[1] - A[1]]]) / 2.0
    det2 = abs(np.linalg.det(J2))
    Gi = np.linalg.inv(J2) @ np.linalg.inv(J2).T * det2     # |det| J^-1 J^-T
    S = Gi[0, 0] * Srr + Gi[0, 1] * (Srs + Srs.T) + Gi[1, 1] * Sss
    return Cc.T @ S @ Cc, det2 * (Cc.T @ Mm @ Cc)


@pytest.mark.parametrize("p", [1, 2, 3, 4])
def test_flat_prism_equals_exact_kronecker_form(p):
    v, t = W.triangulated_box(2, 2, 1.5, 1.0, jitter=0.3, seed=3)
    tm = P.TriMesh(v, t, p)
    nz, h0 = 3, 0.7
    pm = P.PrismMesh(tm, nz)
    eta, h = np.zeros(tm.ns), np.full(tm.ns, h0)
    rule = gll.Rule(p)
    S1 = rule.D.T @ np.diag(rule.w) @ rule.D                  # exact 1D stiffness (degree 2p-2)
    zt = h0 / (2 * nz)
    for e in range(len(t)):
        ST, MT = exact_triangle_matrices(p, *v[t[e]])
        K = np.kron(np.diag(rule.w) * zt, ST) + np.kron(S1 / zt, MT)
        for lay in (0, nz - 1):
            Ke = pm.element_matrix(e, lay, eta, h)
            assert np.max(np.abs(Ke - K)) <= 1e-12 * np.max(np.abs(K))


def curved_case(p, nx=3, nz=2, h0=0.6, amp=0.05):
    v, t = W.triangulated_box(nx, nx, 1.0, 1.0)
    tm = P.TriMesh(v, t, p)
    pm = P.PrismMesh(tm, nz)
    x, y = tm.xs, tm.ys
    eta = amp * np.cos(math.pi * x) * np.sin(0.5 * math.pi * y)
    h = h0 - 0.1 * np.exp(-((x - 0.5) ** 2 + (y - 0.4) ** 2) / 0.05)
    return tm, pm, eta, h


@pytest.mark.parametrize("p", [1, 2, 3])
def test_assembled_operator_properties(p):
    tm, pm, eta, h = curved_case(p, nx=2)
    A = pm.assemble(eta, h).toarray()
    assert np.max(np.abs(A - A.T)) <= 1e-12 * np.max(np.abs(A))
    assert np.max(np.abs(A @ np.ones(pm.N))) <= 1e-11 * np.max(np.abs(A))
    ev = np.linalg.eigvalsh(A)
    assert ev[0] >= -1e-10 * ev[-1] and ev[1] > 1e-8 * ev[-1]   # one zero eigenvalue (constants), the rest > 0


def test_constant_potential_reproduced():
    tm, pm, eta, h = curved_case(3)
    phi = P.laplace_solve(pm, eta, h, np.full(tm.ns, 2.5))
    assert np.max(np.abs(phi - 2.5)) < 1e-12
    assert np.max(np.abs(P.w_recovery(pm, eta, h, phi))) < 1e-11


def dtn_error(nx, p, nz, h0=0.5, amp=0.0):
    """Relative max error of w for cosh(kappa (z + h)) cos(pi x) cos(pi y) in
    the walled unit box (zero normal derivative on every wall and the bottom)."""
    v, t = W.triangulated_box(nx, nx, 1.0, 1.0)
    tm = P.TriMesh(v, t, p)
    pm = P.PrismMesh(tm, nz)
    kx = ky = math.pi
    kap = math.hypot(kx, ky)
    x, y = tm.xs, tm.ys
    eta = amp * np.cos(kx * x) * np.cos(ky * y)
    h = np.full(tm.ns, h0)
    phis = np.cosh(kap * (eta + h0)) * np.cos(kx * x) * np.cos(ky * y)
    w = P.w_recovery(pm, eta, h, P.laplace_solve(pm, eta, h, phis))
    wex = kap * np.sinh(kap * (eta + h0)) * np.cos(kx * x) * np.cos(ky * y)
    return np.max(np.abs(w - wex)) / np.max(np.abs(wex))


def test_dtn_converges_exponentially_in_p():
    errs = [dtn_error(3, p, 2) for p in (1, 2, 3, 4, 5)]
    assert errs[-1] < 5e-4
    assert all(b < 0.35 * a for a, b in zip(errs, errs[1:])), errs
    curved = [dtn_error(3, p, 2, amp=0.03) for p in (2, 3, 4, 5)]
    assert curved[-1] < 1e-3 and all(b < 0.5 * a for a, b in zip(curved, curved[1:])), curved


@pytest.mark.parametrize("p,rate", [(2, 1.7), (3, 2.6)])
def test_dtn_converges_under_refinement(p, rate):
    errs = [dtn_error(nx, p, max(1, nx // 2)) for nx in (2, 4, 8)]
    assert math.log2(errs[1] / errs[2]) > rate, errs


def test_bilinear_form_converges_on_curved_domain():
    """a(I u, I v) = (I u)^T A (I v) for smooth u, v against int grad u . grad v
    over the domain between the bottom z = -h(x, y) (a Gaussian bump) and the
    surface z = eta(x, y), computed by a tensor Gauss rule in (x, y, zeta) with
    z = -h + zeta (eta + h): it converges as p grows (a wrong sign of a
    bathymetry or surface term of the metric does not)."""
    def eta_f(x, y):
        return 0.05 * np.cos(math.pi * x) * np.sin(0.5 * math.pi * y)

    def h_f(x, y):
        return 0.6 - 0.1 * np.exp(-((x - 0.5) ** 2 + (y - 0.4) ** 2) / 0.05)

    def u(x, y, z):
        return np.sin(x + 2 * y) * np.cosh(z)

    def v(x, y, z):
        return np.cos(2 * x - y) * np.exp(z)

    def grads(x, y, z):
        gu = np.stack([np.cos(x + 2 * y) * np.cosh(z), 2 * np.cos(x + 2 * y) * np.cosh(z),
                       np.sin(x + 2 * y) * np.sinh(z)])
        gv = np.stack([-2 * np.sin(2 * x - y) * np.exp(z), np.sin(2 * x - y) * np.exp(z),
                       np.cos(2 * x - y) * np.exp(z)])
        return gu, gv

    g, w = np.polynomial.legendre.leggauss(40)
    g, w = (g + 1) / 2, w / 2
    X, Y, Z = np.meshgrid(g, g, g, indexing="ij")
    WW = w[:, None, None] * w[None, :, None] * w[None, None, :]
    E, H = eta_f(X, Y), h_f(X, Y)
    gu, gv = grads(X, Y, -H + Z * (E + H))
    exact = (WW * (E + H) * (gu * gv).sum(0)).sum()
    errs = []
    for p in (2, 3, 4, 5):
        v_, t_ = W.triangulated_box(3, 3, 1.0, 1.0)
        tm = P.TriMesh(v_, t_, p)
        pm = P.PrismMesh(tm, 2)
        x, y = tm.xs, tm.ys
        eta, h = eta_f(x, y), h_f(x, y)
        xi = pm.rule.xi
        zs = []
        for k in range(pm.nv):
            lay = min(k // p, pm.nz - 1)
            sig = (lay + 0.5 * (1 + xi[k - lay * p])) / pm.nz
            zs.append(-h + sig * (eta + h))
        Zn, Xn, Yn = np.concatenate(zs), np.tile(x, pm.nv), np.tile(y, pm.nv)
        ah = u(Xn, Yn, Zn) @ (pm.assemble(eta, h) @ v(Xn, Yn, Zn))
        errs.append(abs(ah - exact) / abs(exact))
    assert errs[-1] < 1.5e-4 and errs[2] < 3e-4 and errs[-1] < 0.1 * errs[0], errs


# ----------------------------------------------------------------------------- free surface

def test_surface_mass():
    v, t = W.triangulated_box(3, 2, 1.5, 1.0)
    for p in (1, 2, 3):
        pm = P.PrismMesh(P.TriMesh(v, t, p), 1)
        M = P.surface_mass(pm).toarray()
        assert np.max(np.abs(M - M.T)) < 1e-15
        assert abs(M.sum() - 1.5) < 1e-13                      # int 1 dA over the box
        assert np.linalg.eigvalsh(M)[0] > 0
        x, y = pm.tm.xs, pm.tm.ys
        assert abs(x @ M @ np.ones(pm.ns) - 1.5 * 0.75) < 1e-13  # int x dA
        if p >= 2:
            assert abs(x @ M @ x - 1.5 ** 3 / 3.0) < 1e-13       # int x^2 dA, x^2 in the space


def test_projected_conditions_exact_on_the_space():
    """Fields whose free-surface conditions lie in the nodal space are
    reproduced by the projection: eta, phi_eta linear, w linear gives
    f_eta = -grad eta . grad phi + w (1 + |grad eta|^2) linear and
    f_phi = -g eta - |grad phi|^2 / 2 + w^2 (1 + |grad eta|^2) / 2 quadratic."""
    v, t = W.triangulated_box(3, 3, 1.0, 1.0)
    pm = P.PrismMesh(P.TriMesh(v, t, 2), 1)
    x, y = pm.tm.xs, pm.tm.ys
    a, b, c, d, g = 0.03, -0.02, 0.4, 0.7, 9.81
    eta, phis, w = a * x + b * y, c * x + d * y, 0.1 + 0.2 * x - 0.3 * y
    ke, kp = P.project_rhs(pm, eta, phis, w, g)
    q2 = 1 + a * a + b * b
    assert np.max(np.abs(ke - (-(a * c + b * d) + w * q2))) < 1e-13
    assert np.max(np.abs(kp - (-g * eta - 0.5 * (c * c + d * d) + 0.5 * w * w * q2))) < 1e-13
    ke, kp = P.project_rhs(pm, eta, phis, w, g, linear=True)
    assert np.max(np.abs(ke - w)) < 1e-13 and np.max(np.abs(kp + g * eta)) < 1e-13


def standing_wave_error(p, nx=3, nz=2, steps_per_period=24, A=1e-4, h0=0.5, g=9.81):
    """Half a period of the linear standing wave eta = A cos(pi x) cos(omega t)
    in the walled box [0, 2] x [0, 1] (omega^2 = g k tanh(k h), k = pi) on
    triangulated prisms: max error of eta over A."""
    v, t = W.triangulated_box(nx, nx, 2.0, 1.0)
    pm = P.PrismMesh(P.TriMesh(v, t, p), nz)
    k = math.pi
    om = math.sqrt(g * k * math.tanh(k * h0))
    dt = 2 * math.pi / om / steps_per_period
    x = pm.tm.xs
    eta, phis, h = A * np.cos(k * x), np.zeros(pm.ns), np.full(pm.ns, h0)
    n = steps_per_period // 2
    for _ in range(n):
        eta, phis = P.rk4_step(pm, h, eta, phis, dt, g, linear=True)
    return np.max(np.abs(eta - A * np.cos(k * x) * math.cos(om * n * dt))) / A


def test_linear_standing_wave_follows_dispersion_relation():
    """The whole step (prism Laplace solve, w, projected conditions, RK4)
    against the exact linear standing wave; the error falls with p
    (measured 2.0e-1, 8.0e-2, 1.2e-2 for p = 1, 2, 3)."""
    e = [standing_wave_error(p) for p in (1, 2, 3)]
    assert e[2] < 2e-2 and e[2] < 0.25 * e[1] and e[1] < 0.5 * e[0], e


# ----------------------------------------------------------------------------- modal filter

@pytest.mark.parametrize("p", [1, 2, 3, 4, 5])
def test_dubiner_basis_orthonormal(p):
    rq, sq, wq = P.tri_quadrature(p + 2)
    B = P.dubiner(p, rq, sq)
    assert np.max(np.abs(B.T @ (wq[:, None] * B) - np.eye(B.shape[1]))) < 1e-12
    # total degree: psi_(i, j) is a polynomial of degree i + j (the monomial fit of degree i + j is exact)
    for c, (i, j) in enumerate(P.tri_index(p)):
        d = i + j
        M = np.stack([rq ** a * sq ** b for b in range(d + 1) for a in range(d + 1 - b)], 1)
        coef, *_ = np.linalg.lstsq(M, B[:, c], rcond=None)
        assert np.max(np.abs(M @ coef - B[:, c])) < 1e-11


@pytest.mark.parametrize("p", [3, 4, 5])
def test_triangle_filter(p):
    v, t = W.triangulated_box(3, 2, 1.3, 1.0)
    tm = P.TriMesh(v, t, p)
    x, y = tm.xs, tm.ys
    cutoff = 1
    # alpha = 0: the identity
    f = np.sin(3 * x) * np.cos(2 * y)
    assert np.max(np.abs(P.apply_filter(tm, f, 0.0) - f)) < 1e-13
    # polynomials of total degree <= cutoff are unchanged
    lin = 0.3 + 1.2 * x - 0.7 * y
    assert np.max(np.abs(P.apply_filter(tm, lin, 36.0, 4, cutoff) - lin)) < 1e-12
    # one top mode on one triangle: its interior values are scaled by exactly sigma_p
    rn, sn = P.tri_nodes(p)
    top = P.dubiner(p, rn, sn)[:, P.tri_index(p).index((p, 0))]
    Fm = P.filter_matrix(p, 2.0, 2, 0)
    assert np.max(np.abs(Fm @ top - np.exp(-2.0) * top)) < 1e-12
    # a mode of degree d <= p is scaled by sigma_d
    mid = P.dubiner(p, rn, sn)[:, P.tri_index(p).index((1, 1))]
    assert np.max(np.abs(Fm @ mid - np.exp(-2.0 * (2 / p) ** 2) * mid)) < 1e-12


def test_relaxation_step_limits():
    """The prism relaxation step (Sec. 3.3, Step 4.7): C_r = 0 leaves the RK4
    step untouched; C_r = 1 in generation nodes returns exactly the incident
    wave at t + dt (ramped), in absorption nodes exactly zero; a node's blend
    is (1 - C_r) f + C_r f_true with the target at its own position and depth."""
    from oracle import surface as S
    from tests import prism_cases as C
    v, t, pm, h, cr, gen, wave = C.flume(2, 1, nx=4, ny=1)
    eta, h_, phis = C.fields(pm)
    t0, dt = 4.0, 0.02
    e0, p0 = P.rk4_step(pm, h, eta, phis, dt, C.G)
    zero, one = np.zeros(pm.ns), np.ones(pm.ns)
    e1, p1 = P.relaxation_step(pm, h, eta, phis, t0, dt, C.G, zero, one, wave)
    assert np.array_equal(e1, e0) and np.array_equal(p1, p0)
    te, tp = S.incident_wave(pm.tm.xs, pm.tm.ys, h, t0 + dt, g=C.G, **wave)
    e2, p2 = P.relaxation_step(pm, h, eta, phis, t0, dt, C.G, one, one, wave)
    assert np.max(np.abs(e2 - te)) < 1e-15 and np.max(np.abs(p2 - tp)) < 1e-15
    assert abs(np.max(np.abs(te)) - 0.8 * wave["amp"]) < 0.05 * wave["amp"]   # ramp (t + dt) / 5T = 0.804
    e3, p3 = P.relaxation_step(pm, h, eta, phis, t0, dt, C.G, one, zero, wave)
    assert not e3.any() and not p3.any()
    e4, p4 = P.relaxation_step(pm, h, eta, phis, t0, dt, C.G, cr, gen, wave)
    ref_e = np.where(gen != 0, (1 - cr) * e0 + cr * te, (1 - cr) * e0)
    assert np.max(np.abs(e4 - ref_e)) < 1e-15 and np.any((cr > 0) & (cr < 1))


def test_mass_and_energy():
    """Mass and energy of a state on the prism mesh: the mass of eta = c is c
    times the area and that of eta = x its first moment (both exact: the
    fields lie in the space); the energy of a constant elevation at rest is
    g c^2 area / 2; the kinetic energy of the wall mode phi =
    cosh(kap (z + h)) cos(kx x) cos(ky y) on still water (harmonic, zero normal
    derivative on the walls and the bottom) equals, by Green's identity,
    1/2 int phi phi_z dA = kap sinh(kap h) cosh(kap h) Lx Ly / 8, and the
    discrete energy converges to it exponentially in p."""
    import math
    Lx, Ly, h0, g = 1.3, 1.0, 0.5, 9.81
    v, t = W.triangulated_box(3, 2, Lx, Ly)
    kx, ky = math.pi / Lx, math.pi / Ly
    kap = math.hypot(kx, ky)
    exact = kap * math.sinh(kap * h0) * math.cosh(kap * h0) * Lx * Ly / 8
    errs = []
    for p in (2, 3, 4, 5):
        pm = P.PrismMesh(P.TriMesh(v, t, p), 2)
        x, y = pm.tm.xs, pm.tm.ys
        h = np.full(pm.ns, h0)
        assert abs(P.mass(pm, np.full(pm.ns, 0.3)) - 0.3 * Lx * Ly) < 1e-13
        assert abs(P.mass(pm, x) - 0.5 * Lx * Lx * Ly) < 1e-13
        assert abs(P.energy(pm, h, np.full(pm.ns, 0.01), np.zeros(pm.ns), g) - 0.5 * g * 1e-4 * Lx * Ly) < 1e-15
        phis = math.cosh(kap * h0) * np.cos(kx * x) * np.cos(ky * y)
        errs.append(abs(P.energy(pm, h, np.zeros(pm.ns), phis, g) - exact) / exact)
    # measured 5.4e-3, 2.3e-3, 1.1e-4, 5.5e-6 for p = 2..5
    assert all(errs[i + 1] < errs[i] for i in range(len(errs) - 1)), errs
    assert errs[-1] < 1e-5 and errs[-1] < 1e-2 * errs[0], errs


def test_complex_step_derivative_of_the_solve():
    """The prism solve differentiated by a complex step in eta and in h (the
    oracle's arithmetic is analytic: |det J| is written det J sign(Re det J))
    equals central finite differences; real input gives the real solve."""
    from tests import prism_cases as C
    v, t, pm = C.mesh(2, 2, nx=2, ny=1)
    eta, h, phis = C.fields(pm)
    rng = np.random.default_rng(4)
    de, dh = rng.standard_normal(pm.ns), rng.standard_normal(pm.ns)
    eps, fd = 1e-30, 1e-6
    for d_eta, d_h in ((de, 0 * dh), (0 * de, dh)):
        cs = P.laplace_solve(pm, eta + 1j * eps * d_eta, h + 1j * eps * d_h, phis.astype(complex)).imag / eps
        cd = (P.laplace_solve(pm, eta + fd * d_eta, h + fd * d_h, phis)
              - P.laplace_solve(pm, eta - fd * d_eta, h - fd * d_h, phis)) / (2 * fd)
        assert np.linalg.norm(cs - cd) <= 1e-7 * np.linalg.norm(cd)
    real = P.laplace_solve(pm, eta, h, phis)
    zero = P.laplace_solve(pm, eta + 0j, h + 0j, phis)
    assert real.dtype == np.float64 and np.max(np.abs(real - zero.real)) <= 1e-14 * np.max(np.abs(real))
    assert not zero.imag.any()


def test_complex_step_derivative_of_the_rk4_step():
    """One prism RK4 step differentiated by a complex step in (eta, phis) and
    in h equals central finite differences (the whole step's arithmetic is
    analytic: solves, w, projected conditions)."""
    from tests import prism_cases as C
    v, t, pm = C.mesh(2, 2, nx=2, ny=1)
    eta, h, phis = C.fields(pm)
    rng = np.random.default_rng(5)
    de, dp, dh = (rng.standard_normal(pm.ns) for _ in range(3))
    dt, eps, fd = 0.02, 1e-30, 1e-6
    ce, cp = P.rk4_step(pm, h + 1j * eps * dh, eta + 1j * eps * de, phis + 1j * eps * dp, dt, C.G)
    pe, pp = P.rk4_step(pm, h + fd * dh, eta + fd * de, phis + fd * dp, dt, C.G)
    me, mp = P.rk4_step(pm, h - fd * dh, eta - fd * de, phis - fd * dp, dt, C.G)
    for cs, cd in ((ce.imag / eps, (pe - me) / (2 * fd)), (cp.imag / eps, (pp - mp) / (2 * fd))):
        assert np.linalg.norm(cs - cd) <= 1e-6 * np.linalg.norm(cd)
