"""Modal filter of free-surface fields (Sec. 3.2, the modal filtering paragraph).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

On each free-surface element the nodal values g are mapped to the
coefficients of a modal basis, g_hat = V^-1 g, with V_ij = psi_j(r_i) the
Vandermonde matrix of the basis at the element's nodes; a filter matrix F
scales the coefficients and the result is mapped back, V F V^-1 g.

Readings (the paper defines these for its triangles and leaves F to its
reference):
  * quadrilateral surface elements: psi_(a,b)(r, s) = P~_a(r) P~_b(s), the
    tensor products of the orthonormal Legendre polynomials
    P~_k = sqrt((2k + 1) / 2) P_k, at the GLL nodes; in a 2D (x, z) slice the
    surface element is a line and the basis is P~_a(r);
  * F = diag(sigma_a sigma_b) with the exponential filter
    sigma_k = 1 for k <= N_c, exp(-alpha ((k - N_c) / (p - N_c))^s) for k > N_c;
  * the filtered values replace the element-interior nodes only; a node
    shared with a neighbouring element keeps its value (the paper's kernel
    works on the interior point values).
"""
import numpy as np
from numpy.polynomial import legendre as npleg


def vandermonde(rule):
    """V_ij = P~_j(xi_i) on the GLL nodes of the rule."""
    p = rule.p
    V = np.empty((p + 1, p + 1))
    for j in range(p + 1):
        c = np.zeros(j + 1)
        c[j] = 1.0
        V[:, j] = npleg.legval(rule.xi, c) * np.sqrt((2 * j + 1) / 2.0)
    return V


def weights(p, alpha, order, cutoff):
    """sigma_k, k = 0..p, of the exponential filter."""
    k = np.arange(p + 1, dtype=np.float64)
    s = np.ones(p + 1)
    hi = k > cutoff
    s[hi] = np.exp(-alpha * ((k[hi] - cutoff) / (p - cutoff)) ** order)
    return s


def matrix_1d(rule, alpha, order, cutoff):
    """V diag(sigma) V^-1 for one direction."""
    V = vandermonde(rule)
    return V @ np.diag(weights(rule.p, alpha, order, cutoff)) @ np.linalg.inv(V)


def filter_surface(mesh, f, alpha, order, cutoff):
    """Filtered copy of the surface field f [ns]: (F x F) on every surface
    element, written to the element-interior nodes."""
    F = matrix_1d(mesh.rule, alpha, order, cutoff)
    p = mesh.p
    f = np.asarray(f)
    out = f.copy()
    for e in range(mesh.n_ecol):
        cols = mesh.ecol[e]                       # (n, n) in 3D, (n, 1) in 2D
        if mesh.dim == 3:
            gf = F @ f[cols] @ F.T
            out[cols[1:p, 1:p]] = gf[1:p, 1:p]
        else:
            gf = F @ f[cols[:, 0]]
            out[cols[1:p, 0]] = gf[1:p]
    return out
