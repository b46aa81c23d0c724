"""Wave force on a vertical cylinder (oracle, test infrastructure only).

The cylinder configuration's objective (a reading: the paper measures
run-up only): the horizontal force F_x = -int_wall p n_x dS with the pressure
p = -(d phi/dt + 1/2 |grad phi|^2) (Bernoulli, unit density, hydrostatic part
dropped) on the still-water wetted surface of the cylinder r = a,
-h <= z <= 0, n the cylinder's outward normal; over [t_a, t_b]
    J = int n_x (phi(t_b) - phi(t_a)) dS + int_{t_a}^{t_b} int 1/2 |grad phi|^2 n_x dS dt.
Discrete reading: the wall is the row of surface node columns with radial
index 0 of an O-grid mesh; along the wall, the GLL rule of each element edge
with its arc length |d(x, y)/dr|; in z, per element layer l of the
free-surface-following mesh (Sec. 3.1.2; z = -h + sigma (eta + h)) an M_z-point
Gauss-Legendre rule on the part of [-h, 0] the layer covers,
[z_l, z_{l+1}], z_l = -h + (l / N_z)(eta + h), the top layer up to z = 0 (above
a trough its polynomial is evaluated beyond the surface), so the integrand is
smooth on every segment and the segments move smoothly with eta; phi and
grad phi = J^-T grad_(r,s,t) phi (J = d(x, y, z)/d(r, s, t)) are those of the
layer's element; the time integral is the trapezoidal rule.
Written with plain numpy operations that also run on complex numbers, so the
complex-step tangent-linear model differentiates it.
"""
import numpy as np

from .solve import laplace_solve
from . import surface


def _lagrange_deriv(xl, x):
    """d/dx of the cardinal polynomials on nodes xl at the points x (any shape,
    real or complex): [..., n]."""
    n = len(xl)
    out = []
    for j in range(n):
        s = np.zeros_like(x)
        for r in range(n):
            if r == j:
                continue
            term = np.ones_like(x) / (xl[j] - xl[r])
            for m in range(n):
                if m != j and m != r:
                    term = term * (x - xl[m]) / (xl[j] - xl[m])
            s = s + term
        out.append(s)
    return np.stack(out, -1)


def _lagrange_vals(xl, x):
    n = len(xl)
    out = []
    for j in range(n):
        v = np.ones_like(x)
        for m in range(n):
            if m != j:
                v = v * (x - xl[m]) / (xl[j] - xl[m])
        out.append(v)
    return np.stack(out, -1)


def wall_functionals(mesh, eta, h, phi, Mz=8):
    """(P, K): P = int n_x phi dS, K = int 1/2 |grad phi|^2 n_x dS over the
    still-water wetted surface of the radial-index-0 wall of an O-grid mesh
    (3D, periodic in x, walls in y), for the state eta, depth h [Ns] and the
    volume potential phi [N]."""
    p, n, nz, ns = mesh.p, mesh.n, mesh.nz, mesh.ns
    xi, wq = mesh.rule.xi, mesh.rule.w
    D = mesh.rule.D
    zeta, omega = np.polynomial.legendre.leggauss(Mz)
    P = 0.0
    K = 0.0
    for ex in range(mesh.nx):
        ec = ex                                   # element column (ex, ey = 0)
        cols = mesh.ecol[ec]                      # [n, n] global columns of the element's nodes (a, b)
        X, Y = mesh.xh[ec], mesh.yh[ec]           # [n, n]
        E, Hh = eta[cols], h[cols]
        for i in range(n):
            c = cols[i, 0]
            xr = D[i] @ X[:, 0]
            yr = D[i] @ Y[:, 0]
            xs = D[0] @ X[i, :]
            ys = D[0] @ Y[i, :]
            det = xr * ys - xs * yr
            er, hr = D[i] @ E[:, 0], D[i] @ Hh[:, 0]
            es, hs = D[0] @ E[i, :], D[0] @ Hh[i, :]
            rad = np.hypot(X[i, 0], Y[i, 0])
            nx_ = X[i, 0] / rad
            ds = wq[i] * np.hypot(xr, yr)
            for lay, q in ((l_, q_) for l_ in range(nz) for q_ in range(Mz)):
                z_lo = -h[c] + lay / nz * (eta[c] + h[c])
                z_hi = -h[c] + (lay + 1) / nz * (eta[c] + h[c]) if lay < nz - 1 else 0.0
                z = z_lo + 0.5 * (zeta[q] + 1.0) * (z_hi - z_lo)
                sig = (z + h[c]) / (eta[c] + h[c])
                t = 2.0 * (sig * nz - lay) - 1.0
                lv = _lagrange_vals(xi, np.asarray(t))
                ld = _lagrange_deriv(xi, np.asarray(t))
                planes = lay * p + np.arange(n)
                # node (a, b, k) of the element layer: phi[plane_k * ns + cols[a, b]]
                val = sum(lv[k] * phi[planes[k] * ns + cols[i, 0]] for k in range(n))
                ft = sum(ld[k] * phi[planes[k] * ns + cols[i, 0]] for k in range(n))
                fr = sum(D[i, a] * sum(lv[k] * phi[planes[k] * ns + cols[a, 0]] for k in range(n))
                         for a in range(n))
                fs = sum(D[0, b] * sum(lv[k] * phi[planes[k] * ns + cols[i, b]] for k in range(n))
                         for b in range(n))
                # J = [[x_r, x_s, 0], [y_r, y_s, 0], [z_r, z_s, z_t]]; grad phi = J^-T (f_r, f_s, f_t)
                zr = -hr + sig * (er + hr)
                zs = -hs + sig * (es + hs)
                zt = (eta[c] + h[c]) / (2.0 * nz)
                J = np.array([[xr, xs, 0.0], [yr, ys, 0.0], [zr, zs, zt]], dtype=np.result_type(zr, float))
                g = np.linalg.solve(J.T, np.array([fr, fs, ft], dtype=J.dtype))
                wgt = ds * omega[q] * 0.5 * (z_hi - z_lo) * nx_
                P = P + wgt * val
                K = K + wgt * 0.5 * (g[0] * g[0] + g[1] * g[1] + g[2] * g[2])
    return P, K


def force_integral(mesh, h, eta0, phis0, dt, g, n_a, n_b, Mz=8, method="direct"):
    """J = int_{t_a}^{t_b} F_x dt for the oracle's RK4 run from (eta0, phis0)
    (t_a = n_a dt, t_b = n_b dt), trapezoidal rule over the steps."""
    eta, phis = eta0, phis0
    J = 0.0
    for n in range(n_b + 1):
        if n >= n_a:
            phi = laplace_solve(mesh, eta, h, phis, method=method)
            P, K = wall_functionals(mesh, eta, h, phi, Mz)
            wgt = (0.5 if n in (n_a, n_b) else 1.0) * dt
            J = J + wgt * K - (P if n == n_a else 0.0) + (P if n == n_b else 0.0)
        if n < n_b:
            eta, phis = surface.rk4_step(mesh, h, eta, phis, dt, g, method=method)
    return J
