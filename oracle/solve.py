"""Laplace solve for the velocity potential and recovery of w (oracle, test
infrastructure only).

Paper Sec. 2, Eq. (Laplace_strong): Laplace's equation with phi = phi_eta on the
free surface, homogeneous Neumann on the bottom and walls, periodicity on
periodic sides; Sec. 3.1.1, Eq. (Laplace_weak) for the discrete problem; Sec.
3.4 Steps 4.2-4.5 for the order of operations.

The discrete problem: with interior unknowns I (every node below the surface
plane) and surface nodes S, solve  A_II phi_I = -A_IS phi_eta.  The oracle
solves it exactly up to round-off: a sparse direct factorisation (SuperLU) by
default, a dense Cholesky factorisation, or plain CG to a tight tolerance,
which must all agree.  Also a Jacobi-preconditioned CG ("pcg") for meshes
too large for the factorisation.

Vertical velocity (Steps 4.4-4.5; reading: the paper leaves the gradient
recovery unspecified): the z-component of grad phi = J^{-T} grad_r phi at each
surface node, computed in every top-layer element containing the node and
averaged with the lumped surface mass weights w_i w_j |det H|.  Because the
mesh is extruded vertically, d/dz phi = phi_t / z_t is the same in every such
element, so the averaging does not change the value.
"""
import numpy as np
import scipy.linalg as sla
import scipy.sparse.linalg as spla

from .operator import Operator, jacobians, local_derivative_ops


def dirichlet_split(mesh, A):
    nI = mesh.n_interior
    A = A.tocsr()
    return A[:nI, :nI], A[:nI, nI:]


def cg(apply, b, x0=None, rtol=1e-14, max_iter=100000, minv=None):
    """Conjugate gradients (Hestenes-Stiefel); optional diagonal preconditioner
    given as the inverse diagonal minv.  Stops when ||r|| <= rtol ||b||."""
    x = np.zeros_like(b) if x0 is None else x0.copy()
    r = b - apply(x)
    z = r if minv is None else minv * r
    p = z.copy()
    rz = r @ z
    bn = np.sqrt(b @ b)
    it = 0
    while np.sqrt(r @ r) > rtol * bn and it < max_iter:
        q = apply(p)
        alpha = rz / (p @ q)
        x += alpha * p
        r -= alpha * q
        z = r if minv is None else minv * r
        rz_new = r @ z
        p = z + (rz_new / rz) * p
        rz = rz_new
        it += 1
    return x, it


def laplace_solve(mesh, eta, h, phis, op=None, method="direct", rtol=1e-14):
    """Full-volume potential phi (length N, plane-major) with phi = phis on the
    surface plane."""
    phis = np.asarray(phis, dtype=np.result_type(np.asarray(phis), np.float64))
    if op is None:
        op = Operator(mesh, eta, h, assemble=(method != "cg_free"))
    nI = mesh.n_interior
    if method == "cg_free":
        def apply_II(v):
            full = np.concatenate([v, np.zeros(mesh.ns, dtype=v.dtype)])
            return op.apply(full)[:nI]
        b = -op.apply(np.concatenate([np.zeros(nI, dtype=phis.dtype), phis]))[:nI]
        phiI, _ = cg(apply_II, b, rtol=rtol)
    else:
        AII, AIS = dirichlet_split(mesh, op.A)
        b = -(AIS @ phis)
        if method == "direct":
            lu = spla.splu(AII.tocsc(), permc_spec="MMD_AT_PLUS_A", diag_pivot_thresh=0.0,
                           options=dict(SymmetricMode=True))
            if np.iscomplexobj(b) and not np.iscomplexobj(AII.data):
                phiI = lu.solve(np.ascontiguousarray(b.real)) + 1j * lu.solve(np.ascontiguousarray(b.imag))
            else:
                phiI = lu.solve(b)
        elif method == "dense":
            c = sla.cho_factor(AII.toarray())
            phiI = sla.cho_solve(c, b)
        elif method == "cg":
            phiI, _ = cg(lambda v: AII @ v, b, rtol=rtol)
        elif method == "pcg":
            phiI, _ = cg(lambda v: AII @ v, b, rtol=rtol, minv=1.0 / AII.diagonal())
        else:
            raise ValueError(method)
    return np.concatenate([phiI, phis])


def horizontal_jacobian(mesh):
    """H[c, i, j] = d(x, y)/d(r, s) at each surface node of element column c
    (2D: the scalar dx/dr, shape (C, n))."""
    D = mesh.rule.D
    if mesh.dim == 3:
        xr = np.einsum("ia,caj->cij", D, mesh.xh)
        xs = np.einsum("jb,cib->cij", D, mesh.xh)
        yr = np.einsum("ia,caj->cij", D, mesh.yh)
        ys = np.einsum("jb,cib->cij", D, mesh.yh)
        return np.stack([np.stack([xr, xs], -1), np.stack([yr, ys], -1)], -2)
    return np.einsum("ia,ca->ci", D, mesh.xh[:, :, 0])


def surface_weights(mesh):
    """W[c, i(, j)] = w_i (w_j) |det H| : lumped GLL surface mass per element node."""
    w = mesh.rule.w
    H = horizontal_jacobian(mesh)
    if mesh.dim == 3:
        return w[None, :, None] * w[None, None, :] * np.abs(np.linalg.det(H))
    return w[None, :] * np.abs(H)


def surface_cols(mesh):
    return mesh.ecol if mesh.dim == 3 else mesh.ecol[:, :, 0]


def lumped_mass(mesh):
    """Assembled lumped surface mass M[col] = sum over element columns of W."""
    M = np.zeros(mesh.ns)
    np.add.at(M, surface_cols(mesh).ravel(), surface_weights(mesh).ravel())
    return M


def vertical_velocity(mesh, eta, h, phi):
    """w[col] = d phi / dz at the free surface (Steps 4.4-4.5)."""
    J = jacobians(mesh, eta, h)
    Dl = local_derivative_ops(mesh)
    C, n, dim = mesh.n_ecol, mesh.n, mesh.dim
    top = slice((mesh.nz - 1) * C, mesh.nz * C)
    Jt = J[top]
    Jinv = np.linalg.inv(Jt)                          # [c, q, a, m] = d r_a / d x_m
    ph = phi[mesh.glob[top]]                          # (C, nl)
    gr = np.stack([ph @ Da.T for Da in Dl], axis=-1)  # (C, nl, dim): d phi / d r_a
    dz = np.einsum("cqa,cqa->cq", Jinv[..., :, dim - 1], gr)
    if dim == 3:
        dz = dz.reshape(C, n, n, n)[..., n - 1]       # top nodes (k = n-1)
    else:
        dz = dz.reshape(C, n, n)[..., n - 1]
    W = surface_weights(mesh)
    cols = surface_cols(mesh)
    num = np.zeros(mesh.ns, dtype=dz.dtype)
    den = np.zeros(mesh.ns)
    np.add.at(num, cols.ravel(), (W * dz).ravel())
    np.add.at(den, cols.ravel(), W.ravel())
    return num / den


def dtn(mesh, eta, h, phis, method="direct"):
    """Dirichlet-to-Neumann map phi_eta -> w_eta (Steps 4.1-4.5)."""
    phi = laplace_solve(mesh, eta, h, phis, method=method)
    return vertical_velocity(mesh, eta, h, phi), phi
