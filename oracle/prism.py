"""Extruded prism elements on an unstructured triangular surface mesh (oracle).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

The paper builds its fluid mesh from a triangular mesh of the free surface,
extruded vertically into N_z layers of prisms whose columns are translated
vertically to follow the free surface (Sec. 3.1.2), with C0 nodal Lagrange
elements of degree p (Sec. 3.1).  This module restates, for those prisms, what
the hexahedral oracle computes: the stiffness operator of the weak Laplace
form (Eq. Laplace_weak) by its quadrature definition, the Dirichlet-Neumann
solve with phi = phi_eta on the surface (Eq. Laplace_strong), the vertical
surface velocity w (Steps 4.4-4.5), the free-surface conditions projected
with the consistent surface mass, and the RK4 step (Sec. 3.2).

Readings (the paper names the element family, not its nodes or quadrature):
  * element space on a prism: the degree-p polynomials on the triangle times
    the degree-p GLL Lagrange basis in the vertical;
  * triangle nodes: the Blyth-Pozrikidis set built from the 1D GLL points
    v_m in [0, 1] -- node (i, j), k = p - i - j, at barycentric coordinates
    lambda_B = (1 + 2 v_i - v_j - v_k) / 3, lambda_C = (1 + 2 v_j - v_i - v_k) / 3
    (Blyth & Pozrikidis, IMA J. Appl. Math. 71, 2006); its edge nodes are the
    GLL points, so neighbouring triangles share them;
  * straight-sided (affine) triangles in (x, y); in the vertical the mesh of
    the hexahedra: z = -h + sigma (eta + h), sigma = (l + (1 + t) / 2) / N_z,
    with eta and h in the triangle's nodal basis;
  * quadrature: a collapsed-coordinate Gauss-Legendre rule on the triangle,
    exact for total degree 2p + 2, times GLL collocation (p + 1 points) in the
    vertical, as for the hexahedra.
Node numbering: surface nodes are the mesh vertices, then p - 1 nodes per
edge (ordered from the lower to the higher vertex number), then the interior
nodes of each triangle; volume node (plane k, surface node c) is k * Ns + c,
the surface plane k = N_z p.
"""
import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import gll


def tri_index(p):
    """Local node list (i, j), i + j <= p, in the order j outer, i inner."""
    return [(i, j) for j in range(p + 1) for i in range(p + 1 - j)]


def tri_nodes(p):
    """Reference-triangle nodes (r, s) of order p on T = {r, s >= -1, r + s <= 0}
    (vertices A = (-1, -1), B = (1, -1), C = (-1, 1))."""
    v = (gll.nodes(p)[0] + 1.0) / 2.0
    r, s = [], []
    for i, j in tri_index(p):
        k = p - i - j
        lb = (1.0 + 2.0 * v[i] - v[j] - v[k]) / 3.0
        lc = (1.0 + 2.0 * v[j] - v[i] - v[k]) / 3.0
        r.append(2.0 * lb - 1.0)
        s.append(2.0 * lc - 1.0)
    return np.array(r), np.array(s)


def tri_quadrature(n):
    """n x n collapsed Gauss-Legendre rule on T: (r, s, w), exact for total
    degree 2n - 2."""
    a, wa = np.polynomial.legendre.leggauss(n)
    r = ((1.0 + a[None, :]) * (1.0 - a[:, None]) / 2.0 - 1.0).ravel()
    s = np.repeat(a, n)
    w = (wa[None, :] * wa[:, None] * (1.0 - a[:, None]) / 2.0).ravel()
    return r, s, w


def _monomials(p, r, s):
    """u^a v^b (u = (1+r)/2, v = (1+s)/2), a + b <= p, and their r- and
    s-derivatives at the points: three [npts, nb] arrays."""
    u, v = (1.0 + np.asarray(r)) / 2.0, (1.0 + np.asarray(s)) / 2.0
    M, Mr, Ms = [], [], []
    for a, b in tri_index(p):
        M.append(u ** a * v ** b)
        Mr.append(0.5 * a * u ** max(a - 1, 0) * v ** b if a > 0 else 0.0 * u)
        Ms.append(0.5 * b * u ** a * v ** max(b - 1, 0) if b > 0 else 0.0 * u)
    return np.stack(M, -1), np.stack(Mr, -1), np.stack(Ms, -1)


def tri_basis(p, r, s):
    """Values and (r, s)-derivatives of the nodal Lagrange basis of order p on
    T at the points (r, s): three [npts, n_t] arrays (the cardinal functions of
    tri_nodes, from the monomial Vandermonde matrix)."""
    rn, sn = tri_nodes(p)
    V = _monomials(p, rn, sn)[0]
    C = np.linalg.inv(V)
    M, Mr, Ms = _monomials(p, r, s)
    return M @ C, Mr @ C, Ms @ C


class TriMesh:
    """Order-p nodal numbering of an unstructured triangular surface mesh."""

    def __init__(self, verts, tris, p):
        self.p = p
        self.verts = np.asarray(verts, dtype=np.float64)
        self.tris = np.asarray(tris, dtype=np.int64)
        nv = len(self.verts)
        idx = tri_index(p)
        self.nt_loc = len(idx)
        edges = {}
        for t in self.tris:
            for u, w in ((t[0], t[1]), (t[1], t[2]), (t[0], t[2])):
                key = (min(u, w), max(u, w))
                if key not in edges:
                    edges[key] = nv + len(edges) * (p - 1)
        n = nv + len(edges) * (p - 1)
        nodes = np.zeros((len(self.tris), self.nt_loc), dtype=np.int64)
        for e, (A, B, C) in enumerate(self.tris):
            for q, (i, j) in enumerate(idx):
                k = p - i - j
                if (i, j) == (0, 0):
                    g = A
                elif (i, j) == (p, 0):
                    g = B
                elif (i, j) == (0, p):
                    g = C
                elif j == 0:                      # edge A -> B, GLL index i from A
                    g = self._edge(edges, A, B, i)
                elif k == 0:                      # edge B -> C, GLL index j from B
                    g = self._edge(edges, B, C, j)
                elif i == 0:                      # edge A -> C, GLL index j from A
                    g = self._edge(edges, A, C, j)
                else:
                    g = n
                    n += 1
                nodes[e, q] = g
        self.nodes = nodes
        self.ns = n
        rn, sn = tri_nodes(p)
        xs = np.zeros(n)
        ys = np.zeros(n)
        for e, (A, B, C) in enumerate(self.tris):
            lb, lc = (1.0 + rn) / 2.0, (1.0 + sn) / 2.0
            la = 1.0 - lb - lc
            P = la[:, None] * self.verts[A] + lb[:, None] * self.verts[B] + lc[:, None] * self.verts[C]
            xs[nodes[e]] = P[:, 0]
            ys[nodes[e]] = P[:, 1]
        self.xs, self.ys = xs, ys

    def _edge(self, edges, u, w, m):
        p = self.p
        base = edges[(min(u, w), max(u, w))]
        mm = m if u < w else p - m
        return base + mm - 1


class PrismMesh:
    """N_z layers of order-p prisms over a TriMesh."""

    def __init__(self, tm, nz):
        self.tm, self.p, self.nz = tm, tm.p, nz
        self.n = tm.p + 1
        self.rule = gll.Rule(tm.p)
        self.ns = tm.ns
        self.nv = nz * tm.p + 1
        self.N = self.nv * self.ns
        rq, sq, wq = tri_quadrature(tm.p + 2)
        self.wq = wq
        self.L, self.Lr, self.Ls = tri_basis(tm.p, rq, sq)

    def element_matrix(self, e, lay, eta, h):
        """Stiffness matrix [n_t (p+1)]^2 of prism (triangle e, layer lay); local
        node (q, m) -> row m * n_t + q (triangle node q, vertical GLL node m)."""
        tm, p, nz = self.tm, self.p, self.nz
        nt = tm.nt_loc
        A, B, C = tm.verts[tm.tris[e]]
        xr, xs_ = (B[0] - A[0]) / 2.0, (C[0] - A[0]) / 2.0
        yr, ys_ = (B[1] - A[1]) / 2.0, (C[1] - A[1]) / 2.0
        cols = tm.nodes[e]
        E, H = eta[cols], h[cols]
        e_q, er, es = self.L @ E, self.Lr @ E, self.Ls @ E
        h_q, hr, hs = self.L @ H, self.Lr @ H, self.Ls @ H
        xi, wv, D = self.rule.xi, self.rule.w, self.rule.D
        K = np.zeros((nt * (p + 1), nt * (p + 1)), dtype=np.result_type(eta, h, float))
        for k in range(p + 1):
            sig = (lay + 0.5 * (1.0 + xi[k])) / nz
            for q in range(len(self.wq)):
                zr = -hr[q] + sig * (er[q] + hr[q])
                zs = -hs[q] + sig * (es[q] + hs[q])
                zt = (e_q[q] + h_q[q]) / (2.0 * nz)
                J = np.array([[xr, xs_, 0.0], [yr, ys_, 0.0], [zr, zs, zt]])
                det = np.linalg.det(J)
                Jinv = np.linalg.inv(J)
                # reference gradients of every local basis function at (q, t_k)
                gref = np.zeros((3, nt * (p + 1)))
                for m in range(p + 1):
                    sl = slice(m * nt, (m + 1) * nt)
                    if m == k:
                        gref[0, sl] = self.Lr[q]
                        gref[1, sl] = self.Ls[q]
                    gref[2, sl] = self.L[q] * D[k, m]
                g = Jinv.T @ gref
                # |det J| written as det J sign(Re det J): the same value for real
                # input, and analytic, so that a complex step differentiates it
                K += self.wq[q] * wv[k] * (det * np.sign(det.real)) * (g.T @ g)
        return K

    def local_to_global(self, e, lay):
        tm, p, ns = self.tm, self.p, self.ns
        return np.concatenate([(lay * p + m) * ns + tm.nodes[e] for m in range(p + 1)])

    def assemble(self, eta, h):
        """The global stiffness matrix A(eta) [N, N] (scipy CSR)."""
        rows, cols, vals = [], [], []
        for e in range(len(self.tm.tris)):
            for lay in range(self.nz):
                K = self.element_matrix(e, lay, eta, h)
                gi = self.local_to_global(e, lay)
                rows.append(np.repeat(gi, len(gi)))
                cols.append(np.tile(gi, len(gi)))
                vals.append(K.ravel())
        return sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                             shape=(self.N, self.N))


def laplace_solve(pm, eta, h, phis):
    """phi [N] with phi = phis on the surface plane and A_II phi_I = -A_IS phis
    (homogeneous Neumann on the bottom and the lateral walls)."""
    A = pm.assemble(eta, h)
    NI = pm.N - pm.ns
    phi = np.zeros(pm.N, dtype=np.result_type(eta, h, phis, float))
    phi[NI:] = phis
    rhs = -(A[:NI, NI:] @ phis)
    phi[:NI] = spla.spsolve(A[:NI, :NI].tocsc(), rhs)
    return phi


def w_recovery(pm, eta, h, phi):
    """w = d phi / dz at every surface node: phi_t / z_t on its vertical GLL
    line in the top layer (the extrusion is vertical, so every prism sharing
    the line gives this value)."""
    p, ns, nz = pm.p, pm.ns, pm.nz
    D = pm.rule.D
    top = np.stack([phi[(pm.nv - 1 - p + m) * ns:(pm.nv - p + m) * ns] for m in range(p + 1)])
    return (D[p] @ top) * 2.0 * nz / (eta + h)


# ----------------------------------------------------------------------------- free surface
# The free-surface conditions on the triangular surface mesh.  Reading: the
# paper solves its free-surface weak forms with the consistent mass
# (Sec. 3.1.1, Eq. free_surface_weak; Sec. 4 solver settings); here each RHS
# is the Galerkin projection M k = int f l_i dA onto the continuous nodal
# space, f evaluated at the triangle quadrature points from the interpolants of
# eta, phi_eta and w and the element gradients of eta and phi_eta.

def surface_mass(pm):
    """Consistent mass matrix M_ij = int l_i l_j dA of the surface space [Ns, Ns]."""
    tm = pm.tm
    rows, cols, vals = [], [], []
    for e, (A, B, C) in enumerate(tm.tris):
        va, vb, vc = tm.verts[A], tm.verts[B], tm.verts[C]
        det2 = abs((vb[0] - va[0]) * (vc[1] - va[1]) - (vc[0] - va[0]) * (vb[1] - va[1])) / 4.0
        Me = (pm.L * (pm.wq * det2)[:, None]).T @ pm.L
        gi = tm.nodes[e]
        rows.append(np.repeat(gi, len(gi)))
        cols.append(np.tile(gi, len(gi)))
        vals.append(Me.ravel())
    return sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))), shape=(pm.ns, pm.ns))


def project_rhs(pm, eta, phis, w, g, linear=False):
    """(k_eta, k_phi): the Galerkin projections of the kinematic and dynamic
    free-surface conditions (Sec. 2)
        f_eta = -grad eta . grad phi_eta + w (1 + |grad eta|^2)
        f_phi = -g eta - 1/2 |grad phi_eta|^2 + 1/2 w^2 (1 + |grad eta|^2)
    (linear: f_eta = w, f_phi = -g eta)."""
    tm = pm.tm
    dt_ = np.result_type(eta, phis, w, float)   # complex for a complex step
    b_eta = np.zeros(pm.ns, dtype=dt_)
    b_phi = np.zeros(pm.ns, dtype=dt_)
    for e, (A, B, C) in enumerate(tm.tris):
        va, vb, vc = tm.verts[A], tm.verts[B], tm.verts[C]
        J2 = np.array([[vb[0] - va[0], vc[0] - va[0]], [vb[1] - va[1], vc[1] - va[1]]]) / 2.0
        Jit = np.linalg.inv(J2).T
        det2 = abs(np.linalg.det(J2))
        gi = tm.nodes[e]
        E, F, Wn = eta[gi], phis[gi], w[gi]
        eq, wq = pm.L @ E, pm.L @ Wn
        ge = Jit @ np.stack([pm.Lr @ E, pm.Ls @ E])          # [2, nq] physical gradients
        gp = Jit @ np.stack([pm.Lr @ F, pm.Ls @ F])
        if linear:
            fe, fp = wq, -g * eq
        else:
            q2 = 1.0 + (ge * ge).sum(0)
            fe = -(ge * gp).sum(0) + wq * q2
            fp = -g * eq - 0.5 * (gp * gp).sum(0) + 0.5 * wq * wq * q2
        wt = pm.wq * det2
        b_eta[gi] += pm.L.T @ (wt * fe)
        b_phi[gi] += pm.L.T @ (wt * fp)
    M = surface_mass(pm).tocsc()
    return spla.spsolve(M, b_eta), spla.spsolve(M, b_phi)


def rhs(pm, h, eta, phis, g, linear=False):
    """The free-surface right-hand side at (eta, phi_eta): Laplace solve on the
    eta-following prisms (on the still-water mesh when linear), w, projected
    conditions."""
    geo = np.zeros_like(eta) if linear else eta
    phi = laplace_solve(pm, geo, h, phis)
    w = w_recovery(pm, geo, h, phi)
    return project_rhs(pm, eta, phis, w, g, linear)


def rk4_step(pm, h, eta, phis, dt, g, linear=False):
    """One classical RK4 step (Sec. 3.2) of (eta, phi_eta)."""
    k1 = rhs(pm, h, eta, phis, g, linear)
    k2 = rhs(pm, h, eta + 0.5 * dt * k1[0], phis + 0.5 * dt * k1[1], g, linear)
    k3 = rhs(pm, h, eta + 0.5 * dt * k2[0], phis + 0.5 * dt * k2[1], g, linear)
    k4 = rhs(pm, h, eta + dt * k3[0], phis + dt * k3[1], g, linear)
    return (eta + dt / 6.0 * (k1[0] + 2 * k2[0] + 2 * k3[0] + k4[0]),
            phis + dt / 6.0 * (k1[1] + 2 * k2[1] + 2 * k3[1] + k4[1]))


def mass(pm, eta):
    """M = int eta dA over the surface (the consistent surface mass, 1^T M eta)."""
    return float(np.ones(pm.ns) @ (surface_mass(pm) @ eta))


def energy(pm, h, eta, phis, g, linear=False):
    """E = 1/2 phi^T A phi + 1/2 g eta^T M eta (unit density), phi the Laplace
    solution with phi = phis on the surface and A the stiffness matrix of the
    model's geometry (still water when linear)."""
    geo = np.zeros_like(eta) if linear else eta
    phi = laplace_solve(pm, geo, h, phis)
    A = pm.assemble(geo, h)
    return 0.5 * float(phi @ (A @ phi)) + 0.5 * g * float(eta @ (surface_mass(pm) @ eta))


def relaxation_step(pm, h, eta, phis, t, dt, g, cr, gen, wave, linear=False, filt=None):
    """One RK4 step, then the relaxation-zone blend f <- (1 - C_r) f + C_r f_true
    toward the linear incident wave where gen = 1 and toward zero where gen = 0,
    with the targets at t + dt (Sec. 3.3, Step 4.7), at the surface nodes of the
    triangle mesh; then the modal filter of eta and phi_eta when
    filt = (alpha, order, cutoff) (after the relaxation, as on the quadrilateral
    surfaces)."""
    from . import surface as S
    eta, phis = rk4_step(pm, h, eta, phis, dt, g, linear)
    te, tp = S.incident_wave(pm.tm.xs, pm.tm.ys, h, t + dt, g=g, **wave)
    te = np.where(gen != 0, te, 0.0)
    tp = np.where(gen != 0, tp, 0.0)
    eta, phis = S.relax(eta, te, cr), S.relax(phis, tp, cr)
    if filt is not None:
        eta, phis = apply_filter(pm.tm, eta, *filt), apply_filter(pm.tm, phis, *filt)
    return eta, phis


# ----------------------------------------------------------------------------- modal filter
# The paper's modal filter on its triangular surface elements (Sec. 3.2): the
# nodal values of an element are mapped to a modal basis on the reference
# triangle R = {r, s >= -1, r + s <= 0}, g_hat = V^-1 g with V_ij = psi_j(r_i),
# scaled by F and mapped back, V F V^-1 g.  Readings: psi_(i, j) the
# orthonormal Dubiner (PKDO) basis on R; F = diag(sigma_(i+j)) with the
# exponential weights of the quadrilateral filter by total degree,
# sigma_d = 1 for d <= N_c and exp(-alpha ((d - N_c) / (p - N_c))^s) above;
# the filtered values replace the element-interior nodes only (shared nodes
# keep theirs), as for the quadrilaterals.

def _jacobi_normalized(n, a, b, x):
    """The Jacobi polynomial P_n^(a,b)(x) normalised to unit L2 norm with the
    weight (1 - x)^a (1 + x)^b on [-1, 1]."""
    from math import gamma
    from scipy.special import eval_jacobi
    norm = 2.0 ** (a + b + 1) / (2 * n + a + b + 1) * gamma(n + a + 1) * gamma(n + b + 1) / (
        gamma(n + a + b + 1) * gamma(n + 1))
    return eval_jacobi(n, a, b, x) / np.sqrt(norm)


def dubiner(p, r, s):
    """The orthonormal Dubiner basis psi_(i, j), i + j <= p (tri_index order),
    at the points (r, s) of R: [npts, (p+1)(p+2)/2]."""
    r, s = np.asarray(r, dtype=np.float64), np.asarray(s, dtype=np.float64)
    with np.errstate(divide="ignore", invalid="ignore"):
        a = np.where(np.isclose(s, 1.0), -1.0, 2.0 * (1.0 + r) / (1.0 - s) - 1.0)
    out = []
    for i, j in tri_index(p):
        out.append(np.sqrt(2.0) * _jacobi_normalized(i, 0, 0, a) * _jacobi_normalized(j, 2 * i + 1, 0, s)
                   * (1.0 - s) ** i)
    return np.stack(out, -1)


def filter_matrix(p, alpha, order, cutoff):
    """V F V^-1 on the order-p triangle nodes."""
    rn, sn = tri_nodes(p)
    V = dubiner(p, rn, sn)
    sig = []
    for i, j in tri_index(p):
        d = i + j
        sig.append(1.0 if d <= cutoff else float(np.exp(-alpha * ((d - cutoff) / (p - cutoff)) ** order)))
    return V @ np.diag(sig) @ np.linalg.inv(V)


def apply_filter(tm, f, alpha, order=2, cutoff=0):
    """Filtered copy of the surface field f [Ns]: on every triangle the
    interior nodes take the values of V F V^-1 applied to the element's nodal
    values; vertex and edge nodes keep theirs."""
    p = tm.p
    Fm = filter_matrix(p, alpha, order, cutoff)
    idx = tri_index(p)
    interior = np.array([i > 0 and j > 0 and i + j < p for i, j in idx])
    out = np.array(f, dtype=np.result_type(f, float), copy=True)   # complex for a complex step
    for e in range(len(tm.tris)):
        g = tm.nodes[e]
        out[g[interior]] = (Fm @ f[g])[interior]
    return out
