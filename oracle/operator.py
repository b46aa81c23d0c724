"""Stiffness operator of the Laplace weak form (oracle, test infrastructure only).

Paper Sec. 3.1.1, Eq. (Laplace_weak): a[phi; nu] = <grad phi, grad nu>_Omega.
With the nodal GLL basis phi_a and GLL quadrature at the nodes (reading: the
quadrature is the (p+1)^dim-point GLL rule on every element, the "collocation"
choice of Sec. 3.2), the assembled matrix is

    A_ab = sum_e sum_q  w_q |det J_q| (grad_r phi_a)(q)^T  J_q^{-1} J_q^{-T} (grad_r phi_b)(q)

where J_q = d(x, y, z)/d(r, s, t) at GLL point q, obtained by differentiating the
nodal coordinates with the GLL derivative matrix (isoparametric map), and
grad_r phi_a at the nodes is given by D along each reference axis.  Here the
reference gradient is a sparse matrix P = [P_r; P_s; P_t] from global DOF to
element quadrature points and A = P^T Gdiag P; nothing is sum-factorised.
The 3x3 inverse and determinant are general (numpy.linalg), they do not use the
structure of the vertical extrusion.
"""
import numpy as np
import scipy.sparse as sp


def local_derivative_ops(mesh):
    """Dense reference-derivative matrices on one element's nodes, one per axis."""
    n, D = mesh.n, mesh.rule.D
    I = np.eye(n)
    if mesh.dim == 3:
        return [np.kron(np.kron(D, I), I), np.kron(np.kron(I, D), I), np.kron(np.kron(I, I), D)]
    return [np.kron(D, I), np.kron(I, D)]


def quadrature_weights(mesh):
    w = mesh.rule.w
    if mesh.dim == 3:
        return np.kron(np.kron(w, w), w)
    return np.kron(w, w)


def gradient_operators(mesh):
    """Sparse P_alpha (E*nl x N): nodal values -> reference derivative along axis
    alpha at every element quadrature point."""
    Dl = local_derivative_ops(mesh)
    nl = Dl[0].shape[0]
    E = mesh.E
    ops = []
    for Da in Dl:
        qi, ai = np.nonzero(Da)
        vals = Da[qi, ai]
        rows = (np.arange(E)[:, None] * nl + qi[None, :]).ravel()
        cols = mesh.glob[:, ai].ravel()
        data = np.broadcast_to(vals, (E, len(vals))).ravel()
        ops.append(sp.csr_matrix((data, (rows, cols)), shape=(E * nl, mesh.N)))
    return ops


def jacobians(mesh, eta, h):
    """J[e, q, m, a] = d x_m / d r_a at every element node (isoparametric map:
    the GLL derivative of the nodal coordinates); m runs over (x, z) in 2D."""
    x, y, z = mesh.element_coords(eta, h)
    Dl = local_derivative_ops(mesh)
    coords = [x, z] if mesh.dim == 2 else [x, y, z]
    dim = mesh.dim
    E, nl = x.shape
    J = np.empty((E, nl, dim, dim), dtype=np.result_type(x, y, z))
    for m, c in enumerate(coords):
        for a, Da in enumerate(Dl):
            J[:, :, m, a] = c @ Da.T
    return J


def metric(mesh, eta, h):
    """G[e, q, alpha, beta] = w_q |det J| (J^{-1} J^{-T})_{alpha beta} at every
    element quadrature point, and det J."""
    J = jacobians(mesh, eta, h)
    detJ = np.linalg.det(J)
    Jinv = np.linalg.inv(J)                   # Jinv[..., a, m] = d r_a / d x_m
    wq = quadrature_weights(mesh)
    # |det J| written as det J times its (real) orientation sign, which is the
    # same for real data and stays analytic for the complex-step derivative
    absdet = detJ * np.sign(detJ.real)
    G = np.einsum("eqam,eqbm->eqab", Jinv, Jinv) * (wq[None, :] * absdet)[..., None, None]
    return G, detJ


class Operator:
    """The assembled stiffness matrix for one mesh state (eta, h)."""

    def __init__(self, mesh, eta, h, ops=None, assemble=True):
        self.mesh = mesh
        self.P = ops if ops is not None else gradient_operators(mesh)
        self.G, self.detJ = metric(mesh, eta, h)
        dim = mesh.dim
        self.Gflat = [[self.G[:, :, a, b].ravel() for b in range(dim)] for a in range(dim)]
        self.A = None
        if assemble:
            A = None
            for a in range(dim):
                for b in range(dim):
                    term = self.P[a].T @ sp.diags(self.Gflat[a][b]) @ self.P[b]
                    A = term if A is None else A + term
            self.A = A.tocsr()

    def apply(self, x):
        """y = A x without forming A (same definition, used on large meshes)."""
        dim = self.mesh.dim
        g = [Pb @ x for Pb in self.P]
        y = np.zeros(self.mesh.N, dtype=np.result_type(x, self.G))
        for a in range(dim):
            f = sum(self.Gflat[a][b] * g[b] for b in range(dim))
            y += self.P[a].T @ f
        return y

    def element_matrix(self, e):
        Dl = local_derivative_ops(self.mesh)
        dim = self.mesh.dim
        Ae = 0
        for a in range(dim):
            for b in range(dim):
                Ae = Ae + Dl[a].T @ (self.G[e, :, a, b][:, None] * Dl[b])
        return Ae

    def row(self, i, x):
        """(A x)_i computed from the element matrices of the elements containing
        node i only (used to sample outputs of very large meshes)."""
        es, locs = np.nonzero(self.mesh.glob == i)
        s = 0.0
        for e, a in zip(es, locs):
            Ae = self.element_matrix(e)
            s += Ae[a] @ x[self.mesh.glob[e]]
        return s
