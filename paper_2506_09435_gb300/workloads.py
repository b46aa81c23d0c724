"""Seeded synthetic wave-tank workloads shaped like the paper's cases.

This module only produces inputs (mesh descriptors, bathymetry, initial
surface fields); it holds none of the method's arithmetic, so the CPU oracle
and the CUDA path both consume exactly the same arrays.  Fields are evaluated
at surface-node coordinates that the caller passes in.

Physics used for inputs (not the method):
  * linear dispersion relation omega^2 = g k tanh(k h) (used by the paper for
    linear initial conditions, Sec. 3.3),
  * linear (Airy) wave potential  phi = (g a / omega) cosh(k (z + h)) / cosh(k h) sin(k.x + theta)
    evaluated at z = eta for the free-surface potential,
  * the manufactured harmonic potential phi = cosh(kappa (z + h)) cos(kx x) cos(ky y),
    kappa = |(kx, ky)|, with exact vertical velocity d phi/dz.
Random numbers come from splitmix64 (Steele, Lea, Flood 2014), a counter-based
64-bit generator, so that any implementation can reproduce them.
"""
import math

import numpy as np

G_DEFAULT = 9.81
MASK64 = (1 << 64) - 1


def splitmix64(state):
    """One splitmix64 step: returns (new_state, output)."""
    state = (state + 0x9E3779B97F4A7C15) & MASK64
    z = state
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK64
    return state, z ^ (z >> 31)


def uniform01(seed, n):
    """n doubles in [0, 1) from the top 53 bits of successive splitmix64 outputs."""
    out = np.empty(n)
    s = seed & MASK64
    for i in range(n):
        s, z = splitmix64(s)
        out[i] = (z >> 11) * (1.0 / (1 << 53))
    return out


def omega(k, h, g=G_DEFAULT):
    return math.sqrt(g * k * math.tanh(k * h))


def period(k, h, g=G_DEFAULT):
    return 2 * math.pi / omega(k, h, g)


# ----------------------------------------------------------------------------
# mesh descriptors (plain dicts; both sides build their own mesh from them)

def standing_wave_2d(nx=8, nz=2, p=4, kh=1.0, h=1.0, g=G_DEFAULT):
    """2D (x, z) periodic linear standing-wave tank: L = 2 pi / k."""
    k = kh / h
    return dict(dim=2, nx=nx, ny=1, nz=nz, p=p, periodic_x=True, periodic_y=False,
                Lx=2 * math.pi / k, Ly=1.0, h0=h, k=k, g=g)


def periodic_box_3d(nx=32, ny=32, nz=2, p=6, kh=2.0, L=1.0, g=G_DEFAULT):
    """3D periodic box L x L, flat bottom, one wavelength k0 = 2 pi / L along x."""
    k0 = 2 * math.pi / L
    return dict(dim=3, nx=nx, ny=ny, nz=nz, p=p, periodic_x=True, periodic_y=True,
                Lx=L, Ly=L, h0=kh / k0, k=k0, g=g)


def wavenumber(omega_, h, g=G_DEFAULT):
    """k with omega^2 = g k tanh(k h) (Newton on the dispersion relation)."""
    k = omega_ * omega_ / g
    for _ in range(100):
        f = g * k * math.tanh(k * h) - omega_ * omega_
        df = g * math.tanh(k * h) + g * k * h / math.cosh(k * h) ** 2
        dk = f / df
        k -= dk
        if abs(dk) < 1e-15 * k:
            break
    return k


def bar_flume(nx=256, ny=16, nz=3, p=5, Lx=38.0, Ly=1.0, g=G_DEFAULT):
    """Walled wave flume over a submerged trapezoidal bar (the shape of the
    paper's Beji-Battjes case): depth 0.4 m, a 1:20 slope from x = 14 m up to
    0.1 m at x = 20 m, crest to x = 22 m, a 1:10 slope back to 0.4 m at x = 25 m.
    Incident wave T = 2.02 s, H = 0.02 m; generation zone over the first 8 m,
    absorption zone over the last 8 m."""
    T = 2.02
    om = 2 * math.pi / T
    return dict(dim=3, nx=nx, ny=ny, nz=nz, p=p, periodic_x=False, periodic_y=False, Lx=Lx, Ly=Ly, h0=0.4,
                g=g, T=T, omega=om, k=wavenumber(om, 0.4, g), amp=0.01, zone=8.0)


def bar_depth(x):
    x = np.asarray(x, dtype=np.float64)
    h = np.full_like(x, 0.4)
    up = (x >= 14.0) & (x < 20.0)
    h[up] = 0.4 - (x[up] - 14.0) / 20.0
    h[(x >= 20.0) & (x <= 22.0)] = 0.1
    dn = (x > 22.0) & (x < 25.0)
    h[dn] = 0.1 + (x[dn] - 22.0) / 10.0
    return h


def relaxation_weight(xi):
    """C_r on a zone coordinate xi in [0, 1] (0 at the domain edge, 1 at the
    target side): 1 - (exp(xi^3.5) - 1) / (e - 1)."""
    xi = np.clip(np.asarray(xi, dtype=np.float64), 0.0, 1.0)
    return 1.0 - (np.exp(xi ** 3.5) - 1.0) / (math.e - 1.0)


def flume_zones(desc, x):
    """(C_r, gen) at surface nodes x: generation zone [0, zone], absorption zone
    [Lx - zone, Lx]."""
    zone, Lx = desc["zone"], desc["Lx"]
    cr = np.zeros_like(x)
    gen = np.zeros_like(x)
    g_ = x <= zone
    cr[g_] = relaxation_weight(x[g_] / zone)
    gen[g_] = 1.0
    a_ = x >= Lx - zone
    cr[a_] = relaxation_weight((Lx - x[a_]) / zone)
    return cr, gen


def flume_wave(desc):
    """Incident-wave parameters of the relaxation (linear wave along +x)."""
    return dict(amp=desc["amp"], kx=desc["k"], ky=0.0, omega=desc["omega"], phase=0.0, ramp_time=5 * desc["T"])


def dof_counts(desc):
    """Global volume and surface node counts of a structured extruded mesh."""
    p = desc["p"]
    ncx = p * desc["nx"] + (0 if desc["periodic_x"] else 1)
    if desc["dim"] == 3:
        ncy = p * desc["ny"] + (0 if desc["periodic_y"] else 1)
    else:
        ncy = 1
    ns = ncx * ncy
    return (p * desc["nz"] + 1) * ns, ns


# ----------------------------------------------------------------------------
# initial surface states at given surface coordinates

def standing_wave_state(desc, x, amp_over_h=1e-4):
    """eta = a cos(k x) with a = amp_over_h * h, phi_eta = 0."""
    a = amp_over_h * desc["h0"]
    return a * np.cos(desc["k"] * x), np.zeros_like(x)


def airy_potential(x, y, eta, a, kvec, theta, h, g):
    kx, ky = kvec
    k = math.hypot(kx, ky)
    w = omega(k, h, g)
    return (g * a / w) * np.cosh(k * (eta + h)) / math.cosh(k * h) * np.sin(kx * x + ky * y + theta)


def airy_plus_spectrum_state(desc, x, y, seed=2, steepness=0.05, pert_rel=1e-3):
    """Airy wave of height H = steepness * L along x plus a seeded Gaussian
    spectrum of small perturbations in both directions.

    Perturbation modes: k_m = 2 pi (mx / Lx, my / Ly) over the half-plane
    (my > 0, or my == 0 and mx > 0) with 1 <= |k_m| / k0 <= 3; amplitude
    proportional to exp(-(|k_m| - k0)^2 / (2 (0.25 k0)^2)); phases uniform in
    [0, 2 pi) from splitmix64(seed); the sum is scaled so that its maximum
    magnitude over the given nodes is pert_rel * H.  Each component's potential
    follows linear theory and is evaluated at z = eta (total elevation)."""
    g, h, k0 = desc["g"], desc["h0"], desc["k"]
    Lx, Ly = desc["Lx"], desc["Ly"]
    H = steepness * Lx
    a0 = H / 2
    modes = []
    mmax = int(math.ceil(3 * k0 * max(Lx, Ly) / (2 * math.pi))) + 1
    for my in range(0, mmax + 1):
        for mx in range(-mmax, mmax + 1):
            if my == 0 and mx <= 0:
                continue
            kv = (2 * math.pi * mx / Lx, 2 * math.pi * my / Ly)
            kk = math.hypot(*kv)
            if k0 <= kk <= 3 * k0 + 1e-12:
                modes.append((kv, math.exp(-((kk - k0) ** 2) / (2 * (0.25 * k0) ** 2))))
    phases = 2 * math.pi * uniform01(seed, len(modes))
    pert = np.zeros_like(x)
    for (kv, amp), th in zip(modes, phases):
        pert += amp * np.cos(kv[0] * x + kv[1] * y + th)
    scale = pert_rel * H / max(np.max(np.abs(pert)), 1e-300)
    eta = a0 * np.cos(k0 * x) + scale * pert
    # eta = a cos(k.x + theta) travels along +k with potential (g a / omega) ... sin(k.x + theta)
    phis = airy_potential(x, y, eta, a0, (k0, 0.0), 0.0, h, g)
    for (kv, amp), th in zip(modes, phases):
        phis = phis + airy_potential(x, y, eta, scale * amp, kv, th, h, g)
    return eta, phis


def ensemble_tanks(n=64, seed=5, nmin=8, nmax=96, pmin=3, pmax=7):
    """Seeded ensemble of independent periodic tanks (L = 1 m boxes, 2 vertical
    elements): per tank nx, ny ~ U{nmin..nmax}, p ~ U{pmin..pmax}, kh ~ U[0.5, 3],
    steepness H/L ~ U[0.01, 0.06], perturbation seed; from splitmix64(seed)."""
    u = uniform01(seed, 6 * n)
    tanks = []
    for i in range(n):
        a = u[6 * i:6 * i + 6]
        nx = nmin + int(a[0] * (nmax - nmin + 1))
        ny = nmin + int(a[1] * (nmax - nmin + 1))
        p = pmin + int(a[2] * (pmax - pmin + 1))
        kh = 0.5 + 2.5 * a[3]
        steep = 0.01 + 0.05 * a[4]
        d = periodic_box_3d(nx=nx, ny=ny, nz=2, p=p, kh=kh)
        d.update(steepness=steep, seed=1000 + i)
        tanks.append(d)
    return tanks


def ogrid_map(theta, s, a=1.0, R=10.0, stretch=2.0):
    """Annulus around a vertical cylinder of radius a out to R: logical
    coordinates (theta in [0, 2 pi), s in [0, 1]) -> (x, y), with radial
    clustering r = a + (R - a) (exp(stretch s) - 1) / (exp(stretch) - 1); theta
    runs clockwise so that the map (theta, s) -> (x, y) keeps a positive
    orientation."""
    r = a + (R - a) * (np.exp(stretch * s) - 1.0) / (math.exp(stretch) - 1.0)
    return r * np.cos(theta), -r * np.sin(theta)


def cylinder_case(nth=64, nr=24, nz=3, p=4, ka=1.0, kh=1.0, a=1.0, Rout=10.0, g=G_DEFAULT):
    """Wave interaction with a bottom-mounted vertical cylinder (O-grid,
    periodic in theta, walls at the cylinder and at R): k a = 1, k h = 1,
    sponge ring 0.8 R .. R."""
    k = ka / a
    return dict(dim=3, nx=nth, ny=nr, nz=nz, p=p, periodic_x=True, periodic_y=False, Lx=2 * math.pi, Ly=1.0,
                a=a, R=Rout, h0=kh / k, k=k, g=g, T=period(k, kh / k, g))


def triangulated_box(nx, ny, Lx=1.0, Ly=1.0, jitter=0.2, seed=7):
    """Unstructured triangulation of the walled box [0, Lx] x [0, Ly] (the
    paper's surface meshes are triangular, Sec. 3.1.2): an (nx+1) x (ny+1)
    vertex lattice whose interior vertices are moved by up to `jitter` of the
    spacing in each direction (splitmix64(seed) draws), each cell cut into two
    triangles along a diagonal chosen by a draw.  Returns (vertices [nv, 2],
    triangles [nt, 3] counter-clockwise)."""
    dx, dy = Lx / nx, Ly / ny
    u = uniform01(seed, 2 * (nx + 1) * (ny + 1) + nx * ny)
    verts = np.zeros(((nx + 1) * (ny + 1), 2))
    for j in range(ny + 1):
        for i in range(nx + 1):
            v = j * (nx + 1) + i
            x, y = i * dx, j * dy
            if 0 < i < nx:
                x += jitter * dx * (2 * u[2 * v] - 1)
            if 0 < j < ny:
                y += jitter * dy * (2 * u[2 * v + 1] - 1)
            verts[v] = (x, y)
    tris = []
    base = 2 * (nx + 1) * (ny + 1)
    for j in range(ny):
        for i in range(nx):
            a, b = j * (nx + 1) + i, j * (nx + 1) + i + 1
            c, d = a + nx + 1, b + nx + 1
            if u[base + j * nx + i] < 0.5:
                tris += [(a, b, d), (a, d, c)]
            else:
                tris += [(a, b, c), (b, d, c)]
    return verts, np.array(tris, dtype=np.int64)


def prism_flume(nx=64, ny=16, Lx=4.0, Ly=1.0, h0=0.4, T=1.0, amp=0.005, p=4, nz=2, seed=3, g=G_DEFAULT):
    """A walled flume on an unstructured triangulation (the paper's prism mesh
    type, Sec. 3.1.2): the jittered triangulation of triangulated_box, depth h0,
    a generation zone over [0, 1] m and an absorption zone over [Lx - 1, Lx]
    (relaxation_weight profiles) for a linear incident wave of period T and
    amplitude amp.  Returns (verts, tris, desc); flume_zones(desc, x) and
    flume_wave(desc) give the zones and the wave."""
    v, t = triangulated_box(nx, ny, Lx, Ly, seed=seed)
    om = 2.0 * math.pi / T
    desc = dict(p=p, nz=nz, h0=h0, g=g, zone=1.0, Lx=Lx, Ly=Ly, nx=nx, ny=ny, amp=amp,
                k=wavenumber(om, h0, g), omega=om, T=T)
    return v, t, desc


def manufactured_potential(x, y, z, h, kx, ky):
    """Harmonic phi = cosh(kappa (z + h)) cos(kx x) cos(ky y) and its d/dz."""
    kap = math.hypot(kx, ky)
    phi = np.cosh(kap * (z + h)) * np.cos(kx * x) * np.cos(ky * y)
    dphidz = kap * np.sinh(kap * (z + h)) * np.cos(kx * x) * np.cos(ky * y)
    return phi, dphidz


# ----------------------------------------------------------------------------
# steady nonlinear travelling waves (stream-function theory)

class StreamFunctionWave:
    """Steady periodic wave of height H and wavelength L = 2 pi / k on depth d,
    travelling in +x with celerity c, by the Fourier approximation method of
    Rienecker and Fenton (J. Fluid Mech. 104, 1981), written here from its
    equations (an input generator and reference solution; not the FNPF method).

    In the frame moving with the wave (X = x - c t), y the height above the
    bed, the stream function is
        psi(X, y) = B_0 y + sum_{j=1..N} B_j sinh(j k y) / cosh(j k d) cos(j k X)
    (the bed y = 0 is the streamline psi = 0) and the velocity potential
        Phi(X, y) = B_0 X + sum_j B_j cosh(j k y) / cosh(j k d) sin(j k X).
    Unknowns: B_0..B_N, the elevations eta_m at X_m = m L / (2N), m = 0..N
    (crest at X = 0), and the constants Q, R.  Equations at every X_m (on
    y = d + eta_m): psi = -Q (kinematic) and 1/2 |grad psi|^2 + g eta_m = R
    (dynamic); plus the mean of eta = 0 (trapezoid rule over a wavelength) and
    eta_0 - eta_N = H.  With no mean current (Stokes' first definition) c = -B_0.
    Solved by Newton's method with a finite-difference Jacobian, stepping the
    height up from H / steps.

    In the fixed frame, phi = Phi(x - c t, y) + c (x - c t) + (c^2 / 2 - R) t
    solves the Bernoulli condition without a constant (d phi/dt + |grad phi|^2 / 2
    + g eta = 0 on the surface), so the surface potential at time t is
        phi_eta(x, t) = sum_j B_j cosh(j k (d + eta)) / cosh(j k d) sin(j k (x - c t))
                        + (c^2 / 2 - R) t,   eta = eta(x - c t).
    """

    def __init__(self, d, L, H, g=G_DEFAULT, N=24, steps=4, tol=1e-13):
        self.d, self.L, self.H, self.g, self.N = float(d), float(L), float(H), float(g), int(N)
        self.k = 2 * math.pi / self.L
        N, k = self.N, self.k
        self.X = np.arange(N + 1) * self.L / (2 * N)
        c0 = math.sqrt(g / k * math.tanh(k * d))
        # unknown vector: eta_0..eta_N, B_0..B_N, Q, R
        x = np.zeros(2 * N + 4)
        for s in range(1, steps + 1):
            Hs = H * s / steps
            if s == 1:
                x[:N + 1] = 0.5 * Hs * np.cos(k * self.X)
                x[N + 1] = -c0
                x[N + 2] = c0 * 0.5 * Hs / math.tanh(k * d)
                x[2 * N + 2] = c0 * d
                x[2 * N + 3] = 0.5 * c0 * c0
            else:
                x[:N + 1] *= Hs / (H * (s - 1) / steps)
            for _ in range(60):
                r = self._residual(x, Hs)
                if np.max(np.abs(r)) < tol * max(1.0, c0 * c0):
                    break
                J = np.empty((r.size, x.size))
                for i in range(x.size):
                    dx = 1e-7 * max(1.0, abs(x[i]))
                    xp, xm = x.copy(), x.copy()
                    xp[i] += dx
                    xm[i] -= dx
                    J[:, i] = (self._residual(xp, Hs) - self._residual(xm, Hs)) / (2 * dx)
                x = x - np.linalg.solve(J, r)
            else:
                raise RuntimeError("stream-function iteration did not converge")
        self.eta_m = x[:N + 1].copy()
        self.B = x[N + 1:2 * N + 2].copy()
        self.Q, self.R = x[2 * N + 2], x[2 * N + 3]
        self.c = -self.B[0]
        self.residual = float(np.max(np.abs(self._residual(x, H))))
        # cosine coefficients of eta(X) interpolating eta_m (DCT-I pair)
        m = np.arange(N + 1)
        w = np.ones(N + 1)
        w[0] = w[N] = 0.5
        self.E = np.array([2.0 / N * np.sum(w * self.eta_m * np.cos(j * m * math.pi / N)) for j in range(N + 1)])

    def _residual(self, x, H):
        N, k, d, g = self.N, self.k, self.d, self.g
        eta, B, Q, R = x[:N + 1], x[N + 1:2 * N + 2], x[2 * N + 2], x[2 * N + 3]
        y = d + eta
        j = np.arange(1, N + 1)[None, :]
        kx = j * k * self.X[:, None]
        sh = np.sinh(j * k * y[:, None]) / np.cosh(j * k * d)
        ch = np.cosh(j * k * y[:, None]) / np.cosh(j * k * d)
        psi = B[0] * y + np.sum(B[1:] * sh * np.cos(kx), axis=1)
        U = B[0] + np.sum(j * k * B[1:] * ch * np.cos(kx), axis=1)
        W = np.sum(j * k * B[1:] * sh * np.sin(kx), axis=1)
        wt = np.ones(N + 1)
        wt[0] = wt[N] = 0.5
        return np.concatenate([psi + Q, 0.5 * (U * U + W * W) + g * eta - R,
                               [np.sum(wt * eta) / N, eta[0] - eta[N] - H]])

    def eta(self, x, t=0.0):
        X = np.asarray(x, dtype=np.float64) - self.c * t
        j = np.arange(self.N + 1)
        w = np.ones(self.N + 1)
        w[0] = w[self.N] = 0.5
        return np.sum(w * self.E * np.cos(j * self.k * X[..., None]), axis=-1)

    def phis(self, x, t=0.0):
        X = np.asarray(x, dtype=np.float64) - self.c * t
        y = self.d + self.eta(x, t)
        j = np.arange(1, self.N + 1)
        ch = np.cosh(j * self.k * y[..., None]) / np.cosh(j * self.k * self.d)
        return np.sum(self.B[1:] * ch * np.sin(j * self.k * X[..., None]), axis=-1) \
            + (0.5 * self.c * self.c - self.R) * t

    def period(self):
        return self.L / self.c


def stream_function_tank_2d(nx=4, nz=2, p=6, kh=1.0, steepness=0.05, h=1.0, g=G_DEFAULT, N=24):
    """2D periodic tank of one wavelength holding a stream-function wave of
    height H = steepness L (the paper's nonlinear convergence studies use
    stream-function waves, Sec. 3.3)."""
    k = kh / h
    L = 2 * math.pi / k
    wave = StreamFunctionWave(h, L, steepness * L, g=g, N=N)
    return dict(dim=2, nx=nx, ny=1, nz=nz, p=p, periodic_x=True, periodic_y=False,
                Lx=L, Ly=1.0, h0=h, k=k, g=g), wave
