"""Objective functionals of the differentiation form (the user's side of a
gradient computation).

A gradient with respect to the initial state or the bathymetry needs an
objective J of the states an RK4 run produces.  This module gives the
objective of the cylinder configuration, the horizontal wave force on a
bottom-mounted vertical cylinder, written with torch operations on the surface
state and on the volume potential of a Laplace solve, so that torch.autograd
differentiates J and hands its cotangents to the library's adjoint:
`LaplaceSolve` wraps fnpf_laplace_solve / fnpf_laplace_solve_vjp and
`autograd.rk4_run` the RK4 steps.  The solves and steps run in libfnpf's
kernels; the functional itself is a small gather-and-sum over the wall.

Force (a reading: the paper's cylinder case reports run-up only):
    F_x(t) = -int_wall p n_x dS,   p = -(d phi/dt + 1/2 |grad phi|^2)
(unit density, hydrostatic part dropped, n the cylinder's outward normal) on
the still-water wetted surface r = a, -h <= z <= 0.  Over [t_a, t_b]
    J = int n_x [phi(t_b) - phi(t_a)] dS + int_{t_a}^{t_b} int 1/2 |grad phi|^2 n_x dS dt,
the d phi/dt part integrated exactly in time on the fixed surface.
Discretely: the wall is the row of surface node columns with radial index 0 of
an O-grid (periodic in the first, walled in the second horizontal direction);
the wall integral takes the GLL weights of the element edges along the wall
times their arc length and, per element layer l of the free-surface-following
mesh (z = -h + sigma (eta + h)), an M_z-point Gauss-Legendre rule on the part
of [-h, 0] the layer covers, [z_l, z_{l+1}] with z_l = -h + (l / N_z)(eta + h),
the top layer up to z = 0 (above a trough its polynomial is evaluated beyond
the surface): the integrand is smooth on every segment and the segments move
smoothly with eta.  phi and its gradient are the layer's element's; the time
integral is the trapezoidal rule over the steps.
"""
import numpy as np
import torch

from .autograd import _check_depth, rk4_trajectory


def _gll(p):
    """GLL nodes (ascending), weights and derivative matrix D[i, a] = l_a'(x_i)
    of order p: Newton iteration on (1 - x^2) P_p'(x) from Chebyshev-Lobatto
    points; weights 2 / (p (p+1) P_p(x)^2); D by differentiating the Lagrange
    cardinal polynomials (sum over the omitted factor)."""
    x = -np.cos(np.pi * np.arange(p + 1) / p)
    for _ in range(100):
        pm, pc = np.ones_like(x), x.copy()
        for k in range(1, p):
            pm, pc = pc, ((2 * k + 1) * x * pc - k * pm) / (k + 1)
        q = p * (pm - x * pc)                 # (1 - x^2) P_p'
        dq = -p * (p + 1) * pc
        dx = np.zeros_like(x)
        dx[1:-1] = q[1:-1] / dq[1:-1]
        x = x - dx
        if np.max(np.abs(dx)) < 1e-16:
            break
    x[0], x[-1] = -1.0, 1.0
    pm, pc = np.ones_like(x), x.copy()
    for k in range(1, p):
        pm, pc = pc, ((2 * k + 1) * x * pc - k * pm) / (k + 1)
    w = 2.0 / (p * (p + 1) * pc * pc)
    n = p + 1
    D = np.zeros((n, n))
    for a in range(n):
        den = np.prod([x[a] - x[m] for m in range(n) if m != a])
        for i in range(n):
            s = 0.0
            for r in range(n):
                if r == a:
                    continue
                s += np.prod([x[i] - x[m] for m in range(n) if m != a and m != r])
            D[i, a] = s / den
    return x, w, D


class WallForce:
    """Wall functionals P(y) = int n_x phi dS and K(y) = int 1/2 |grad phi|^2 n_x dS
    over the still-water wetted surface of the wall at radial index 0 of an
    O-grid mesh, from the surface state (eta, h) and the volume potential phi."""

    def __init__(self, mesh, X, Y, Mz=8, device=None):
        if mesh.dim != 3 or not mesh.periodic_x or mesh.periodic_y:
            raise ValueError("the wall is the radial-index-0 row of a 3D O-grid (periodic x, walls in y)")
        p, n, nx, nz = mesh.p, mesh.p + 1, mesh.nx, mesh.nz
        ncx = p * nx
        xi, w, D = _gll(p)
        X = np.asarray(X, dtype=np.float64)
        Y = np.asarray(Y, dtype=np.float64)
        ex = np.arange(nx)[:, None]
        i = np.arange(n)[None, :]
        colW = (ex * p + i) % ncx                                   # [ex, i]
        colA = np.repeat(colW[:, None, :], n, axis=1)               # [ex, i, a]: node (a, 0) of element ex
        colB = colW[:, :, None] + ncx * np.arange(n)[None, None, :]  # [ex, i, b]: node (i, b)
        xr = np.einsum("ia,eia->ei", D, X[colA])
        yr = np.einsum("ia,eia->ei", D, Y[colA])
        xs = np.einsum("b,eib->ei", D[0], X[colB])
        ys = np.einsum("b,eib->ei", D[0], Y[colB])
        r = np.hypot(X[colW], Y[colW])
        zeta, omega = np.polynomial.legendre.leggauss(Mz)
        dev = device if device is not None else torch.device("cuda", torch.cuda.current_device())
        t = lambda a, dt=torch.float64: torch.as_tensor(np.ascontiguousarray(a), dtype=dt, device=dev)
        self.p, self.n, self.nz, self.ns, self.N = p, n, nz, mesh.ns, mesh.N
        self.xi = t(xi)
        self.D = t(D)
        self.colW, self.colA, self.colB = t(colW, torch.long), t(colA, torch.long), t(colB, torch.long)
        self.xr, self.xs, self.yr, self.ys = t(xr), t(xs), t(yr), t(ys)
        self.det = t(xr * ys - xs * yr)
        self.W = t(w[None, :] * np.hypot(xr, yr))                    # GLL weight x arc length
        self.nxn = t(X[colW] / r)                                   # n_x of the cylinder's outward normal
        self.zeta, self.omega = t(zeta), t(omega)

    def _lagrange(self, s):
        """Values and derivatives of the GLL cardinal polynomials at s [...]: [..., n]."""
        xi, n = self.xi, self.n
        vals, ders = [], []
        for k in range(n):
            v = torch.ones_like(s)
            d = torch.zeros_like(s)
            for m in range(n):
                if m == k:
                    continue
                f = (s - xi[m]) / (xi[k] - xi[m])
                d = d * f + v / (xi[k] - xi[m])
                v = v * f
            vals.append(v)
            ders.append(d)
        return torch.stack(vals, -1), torch.stack(ders, -1)

    def evaluate(self, eta, h, phi):
        """(P, K) for the surface elevation eta [Ns], depth h [Ns] and volume
        potential phi [N] (torch tensors; differentiable in all three)."""
        ns, p, nz, n = self.ns, self.p, self.nz, self.n
        dev = phi.device
        hw, ew = h[self.colW], eta[self.colW]                         # [ex, i]
        lay = torch.arange(nz, device=dev, dtype=torch.float64)
        depth = (ew + hw)[..., None]
        z_lo = -hw[..., None] + lay / nz * depth                     # [ex, i, L]
        z_hi = torch.where(lay < nz - 1, -hw[..., None] + (lay + 1) / nz * depth, torch.zeros_like(z_lo))
        z = z_lo[..., None] + 0.5 * (self.zeta + 1.0) * (z_hi - z_lo)[..., None]     # [ex, i, L, q]
        sig = (z + hw[..., None, None]) / depth[..., None]
        st = 2.0 * (sig * nz - lay[:, None]) - 1.0
        lv, ld = self._lagrange(st)                                  # [ex, i, L, q, k]
        planes = ((torch.arange(nz, device=dev)[:, None] * p + torch.arange(n, device=dev)) * ns)   # [L, k]
        phW = phi[self.colW[:, :, None, None] + planes]              # [ex, i, L, k]
        phA = phi[self.colA[..., None, None] + planes]               # [ex, i, a, L, k]
        phB = phi[self.colB[..., None, None] + planes]               # [ex, i, b, L, k]
        val = (lv * phW[:, :, :, None, :]).sum(-1)                   # [ex, i, L, q]
        dt_ = (ld * phW[:, :, :, None, :]).sum(-1)
        dr = torch.einsum("ia,eialq->eilq", self.D, (lv[:, :, None] * phA[:, :, :, :, None, :]).sum(-1))
        ds = torch.einsum("b,eiblq->eilq", self.D[0], (lv[:, :, None] * phB[:, :, :, :, None, :]).sum(-1))
        er = torch.einsum("ia,eia->ei", self.D, eta[self.colA])
        hr = torch.einsum("ia,eia->ei", self.D, h[self.colA])
        es = torch.einsum("b,eib->ei", self.D[0], eta[self.colB])
        hs = torch.einsum("b,eib->ei", self.D[0], h[self.colB])
        zr = -hr[..., None, None] + sig * (er + hr)[..., None, None]
        zs = -hs[..., None, None] + sig * (es + hs)[..., None, None]
        zt = (depth / (2.0 * nz))[..., None]
        fz = dt_ / zt
        gr, gs = dr - zr * fz, ds - zs * fz
        e4 = lambda a: a[..., None, None]
        fx = (e4(self.ys) * gr - e4(self.yr) * gs) / e4(self.det)
        fy = (-e4(self.xs) * gr + e4(self.xr) * gs) / e4(self.det)
        wq = e4(self.W * self.nxn) * self.omega * (0.5 * (z_hi - z_lo))[..., None]
        P = (wq * val).sum()
        K = (wq * 0.5 * (fx * fx + fy * fy + fz * fz)).sum()
        return P, K


class LaplaceSolve(torch.autograd.Function):
    """phi [N] = fnpf_laplace_solve(eta, phis), differentiable in eta, phis and
    h (through fnpf_laplace_solve_vjp); h must be the mesh's depth."""

    @staticmethod
    def forward(ctx, eta, phis, h, mesh):
        eta_c, phis_c = eta.detach().contiguous(), phis.detach().contiguous()
        phi = torch.zeros(mesh.N, dtype=torch.float64, device=eta.device)
        mesh.laplace_solve(eta_c, phis_c, phi)
        ctx.mesh = mesh
        ctx.save_for_backward(eta_c, phis_c, phi)
        return phi

    @staticmethod
    def backward(ctx, gphi):
        eta, phis, phi = ctx.saved_tensors
        le, lp, lh = torch.zeros_like(eta), torch.zeros_like(eta), torch.zeros_like(eta)
        ctx.mesh.laplace_solve_vjp(eta, phis, phi, gphi.contiguous(), le, lp, lh)
        return le, lp, lh, None


def cylinder_force_objective(mesh, wall, eta0, phis0, h, t0, dt, n_a, n_b, every=16):
    """J = int_{t_a}^{t_b} F_x dt with t_a = t0 + n_a dt, t_b = t0 + n_b dt
    (trapezoidal rule over the steps), as a differentiable torch scalar of the
    initial state (eta0, phis0) and the depth h (the mesh's)."""
    if not 0 <= n_a < n_b:
        raise ValueError("need 0 <= n_a < n_b")
    _check_depth(mesh, h)
    etas, phiss = rk4_trajectory(mesh, eta0, phis0, h, t0, dt, n_b, n_a, every)
    J = None
    for k in range(n_b - n_a + 1):
        P, K = wall.evaluate(etas[k], h, LaplaceSolve.apply(etas[k], phiss[k], h, mesh))
        wgt = (0.5 if k in (0, n_b - n_a) else 1.0) * dt
        term = wgt * K - (P if k == 0 else 0.0) + (P if k == n_b - n_a else 0.0)
        J = term if J is None else J + term
    return J
