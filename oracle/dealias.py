"""Over-integration of the nonlinear free-surface terms (oracle, test
infrastructure only).

Paper Sec. 3.2 (temporal discretization and modal filtering): besides the
modal filter, the nonlinear terms of the free-surface conditions are
integrated with a quadrature of higher order than the nodal collocation, to
reduce the aliasing that destabilises steep waves (the paper sets a higher
integration degree on those terms of its weak forms).  Reading taken here
(the GLL collocation and lumped mass of the rest of the oracle stay):

  * on every surface element the nodal fields eta, phi_eta and w are
    interpolated (their Lagrange interpolants on the GLL nodes) to a
    Gauss-Legendre rule of M points per direction, their horizontal gradients
    are those of the interpolants (the inverse horizontal Jacobian from the
    interpolated node coordinates), and the Zakharov right-hand sides
    f_eta, f_phi of Sec. 2 are evaluated at those points;
  * each is replaced by its L2 projection onto the tensor polynomials of
    degree p in the element's reference coordinates, computed exactly by the
    Gauss rule (Legendre coefficients c_k = sum_q w_q f(r_q) P_k(r_q) / gamma_k,
    gamma_k = 2 / (2k + 1)) and evaluated at the GLL nodes;
  * the element values at shared nodes are combined with the lumped-mass
    weights W_e = w_i w_j |det H| as the collocation right-hand side is.

A right-hand side that is itself a polynomial of degree <= p in each
reference direction is reproduced exactly (as collocation does), so linear
terms are unchanged; products of higher degree lose the modes above p instead
of folding them onto the nodes.
"""
import numpy as np

from .gll import derivative_matrix, lagrange_eval, legendre, nodes
from .solve import lumped_mass, surface_cols, surface_weights


def gauss_rule(M):
    """Gauss-Legendre points and weights on [-1, 1] (numpy's Golub-Welsch)."""
    return np.polynomial.legendre.leggauss(M)


def projection_matrix(p, M):
    """Pi [n x M]: values at the GLL nodes of the L2 projection onto P_p of a
    function sampled at the M Gauss points."""
    xq, wq = gauss_rule(M)
    xi = nodes(p)[0]
    Lq = np.stack([legendre(k, xq)[0] for k in range(p + 1)], axis=1)    # [M, n]: P_k(x_q)
    V = np.stack([legendre(k, xi)[0] for k in range(p + 1)], axis=1)     # [n, n]: P_k(xi_i)
    gamma = 2.0 / (2 * np.arange(p + 1) + 1.0)
    return V @ np.diag(1.0 / gamma) @ Lq.T @ np.diag(wq)


def interpolation_matrices(p, M):
    """B [M x n] (values) and Bd [M x n] (derivatives) of the GLL Lagrange
    basis at the Gauss points.  Bd = B D: the derivative of a degree-p
    interpolant is a polynomial of degree p - 1, reproduced by its GLL
    interpolant."""
    xq, _ = gauss_rule(M)
    B = lagrange_eval(nodes(p)[0], xq)
    return B, B @ derivative_matrix(p)


def zakharov_rhs_dealiased(mesh, eta, phis, w, g, M):
    """(d eta/dt, d phi_eta/dt) at every surface column, with the nonlinear
    terms over-integrated on M Gauss points per direction."""
    p = mesh.p
    B, Bd = interpolation_matrices(p, M)
    Pi = projection_matrix(p, M)
    cols = surface_cols(mesh)
    E, F, Wn = eta[cols], phis[cols], w[cols]
    if mesh.dim == 3:
        def at_q(A, Br, Bs):                       # [C, n, n] -> [C, M, M]
            return np.einsum("qa,cab,rb->cqr", Br, A, Bs)
        X, Y = mesh.xh, mesh.yh
        xr, xs = at_q(X, Bd, B), at_q(X, B, Bd)
        yr, ys = at_q(Y, Bd, B), at_q(Y, B, Bd)
        det = xr * ys - xs * yr
        # grad f = J^-T (f_r, f_s) with J = [[x_r, x_s], [y_r, y_s]]
        def grad(A):
            fr, fs = at_q(A, Bd, B), at_q(A, B, Bd)
            return (ys * fr - yr * fs) / det, (-xs * fr + xr * fs) / det
        ex, ey = grad(E)
        px, py = grad(F)
        eq, wq = at_q(E, B, B), at_q(Wn, B, B)
        ge2 = ex * ex + ey * ey
        fe = -(ex * px + ey * py) + wq * (1 + ge2)
        fp = -g * eq - 0.5 * (px * px + py * py) + 0.5 * wq * wq * (1 + ge2)
        fe_n = np.einsum("iq,cqr,jr->cij", Pi, fe, Pi)
        fp_n = np.einsum("iq,cqr,jr->cij", Pi, fp, Pi)
    else:
        X = mesh.xh[:, :, 0]
        xr = np.einsum("qa,ca->cq", Bd, X)
        ex = np.einsum("qa,ca->cq", Bd, E) / xr
        px = np.einsum("qa,ca->cq", Bd, F) / xr
        eq = np.einsum("qa,ca->cq", B, E)
        wq = np.einsum("qa,ca->cq", B, Wn)
        ge2 = ex * ex
        fe = -ex * px + wq * (1 + ge2)
        fp = -g * eq - 0.5 * px * px + 0.5 * wq * wq * (1 + ge2)
        fe_n = np.einsum("iq,cq->ci", Pi, fe)
        fp_n = np.einsum("iq,cq->ci", Pi, fp)
    W = surface_weights(mesh)
    Ml = lumped_mass(mesh)
    d_eta = np.zeros(mesh.ns, dtype=fe_n.dtype)
    d_phi = np.zeros(mesh.ns, dtype=fp_n.dtype)
    np.add.at(d_eta, cols.ravel(), (W * fe_n).ravel())
    np.add.at(d_phi, cols.ravel(), (W * fp_n).ravel())
    return d_eta / Ml, d_phi / Ml


def rk4_step_dealiased(mesh, h, eta, phis, dt, g, M, method="direct"):
    """One classical RK4 step (Sec. 3.2) with the over-integrated right-hand side."""
    from .solve import dtn

    def F(e, p_):
        wv, _ = dtn(mesh, e, h, p_, method=method)
        return zakharov_rhs_dealiased(mesh, e, p_, wv, g, M)
    k1 = F(eta, phis)
    k2 = F(eta + 0.5 * dt * k1[0], phis + 0.5 * dt * k1[1])
    k3 = F(eta + 0.5 * dt * k2[0], phis + 0.5 * dt * k2[1])
    k4 = F(eta + dt * k3[0], phis + dt * k3[1])
    return (eta + dt / 6 * (k1[0] + 2 * k2[0] + 2 * k3[0] + k4[0]),
            phis + dt / 6 * (k1[1] + 2 * k2[1] + 2 * k3[1] + k4[1]))
