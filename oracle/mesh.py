"""Extruded structured mesh following the free surface (oracle, test infrastructure only).

Follows the paper's mesh construction (Sec. 3.1.2): a horizontal surface mesh
is extruded vertically into N_z layers, and every column of points is then
translated vertically so that the top follows eta and the bottom follows the
bathymetry z = -h (Step 4.1 of Sec. 3.4).  Readings taken where the paper is
silent:
  * quadrilateral/hexahedral elements with tensor GLL nodes (the paper uses
    triangles/prisms; node counts of the periodic meshes coincide),
  * uniform layers: z = -h + sigma (eta + h), sigma = (l + (1 + xi_k)/2) / N_z
    in layer l (the paper only says "vertical translation along each column").

Node numbering ("plane-major"): global index = k * N_s + col, with k = 0 at the
bottom and k = N_v - 1 = p N_z on the free surface, and col = iy * ncx + ix
(ix fastest).  Periodic directions identify the last node column with the
first.  dim = 2 is the (x, z) vertical slice: there is no y and ncy = 1.
"""
from functools import cached_property

import numpy as np

from .gll import Rule


class Mesh:
    def __init__(self, dim, nx, ny, nz, p, periodic_x=True, periodic_y=True,
                 Lx=1.0, Ly=1.0, X=None, Y=None):
        if dim not in (2, 3):
            raise ValueError("dim must be 2 or 3")
        if dim == 2:
            ny, periodic_y = 1, False
        self.dim, self.nx, self.ny, self.nz, self.p = dim, nx, ny, nz, p
        self.periodic_x, self.periodic_y = bool(periodic_x), bool(periodic_y)
        self.rule = Rule(p)
        n = p + 1
        self.n = n
        self.ncx = p * nx + (0 if periodic_x else 1)
        self.ncy = (p * ny + (0 if periodic_y else 1)) if dim == 3 else 1
        self.ns = self.ncx * self.ncy            # surface (column) count
        self.nv = p * nz + 1                     # nodes per column
        self.N = self.nv * self.ns               # volume DOF
        self.n_interior = (self.nv - 1) * self.ns
        self.Lx, self.Ly = Lx, Ly
        self.iso = X is not None
        if self.iso:
            self.X = np.asarray(X, dtype=np.float64).reshape(self.ns)
            self.Y = np.asarray(Y, dtype=np.float64).reshape(self.ns)

        self.n_ecol = nx * ny
        self.E = self.n_ecol * nz

    @cached_property
    def _arrays(self):
        dim, nx, ny, nz, p, n = self.dim, self.nx, self.ny, self.nz, self.p, self.n
        periodic_x, periodic_y, Lx, Ly = self.periodic_x, self.periodic_y, self.Lx, self.Ly
        # element-column -> global column of each local horizontal node
        ny_loc = n if dim == 3 else 1
        ex = np.arange(nx)[:, None, None, None]
        ey = np.arange(ny)[None, :, None, None]
        i = np.arange(n)[None, None, :, None]
        j = np.arange(ny_loc)[None, None, None, :]
        ix = ex * p + i
        iy = ey * p + j if dim == 3 else 0 * j
        if periodic_x:
            ix = ix % self.ncx
        if dim == 3 and periodic_y:
            iy = iy % self.ncy
        # shape (ny, nx, n, ny_loc): element columns ordered ex fastest
        col = (iy * self.ncx + ix).transpose(1, 0, 2, 3)
        ecol_ = col.reshape(ny * nx, n, ny_loc)      # [ecolumn, i, j]
        n_ecol = nx * ny

        # horizontal coordinates of each element-column node (element-local, so that
        # a periodic element sees x = Lx on its last node, not the wrapped 0)
        xi = self.rule.xi
        if self.iso:
            xh_ = self.X[ecol_]
            yh_ = self.Y[ecol_]
        else:
            dx = Lx / nx
            exx = np.arange(nx)[None, :, None, None]
            xh = exx * dx + (1 + xi)[None, None, :, None] * dx / 2
            xh = np.broadcast_to(xh, (ny, nx, n, ny_loc))
            if dim == 3:
                dy = Ly / ny
                eyy = np.arange(ny)[:, None, None, None]
                yh = eyy * dy + (1 + xi)[None, None, None, :] * dy / 2
                yh = np.broadcast_to(yh, (ny, nx, n, ny_loc))
            else:
                yh = np.zeros((ny, nx, n, ny_loc))
            xh_ = np.ascontiguousarray(xh).reshape(n_ecol, n, ny_loc)
            yh_ = np.ascontiguousarray(yh).reshape(n_ecol, n, ny_loc)

        # volume elements: e = ez * n_ecol + ecolumn; local node order (i, j, k) or (i, k)
        E = n_ecol * nz

        k = np.arange(n)
        glob = []
        for ez in range(nz):
            kg = ez * p + k                               # (n,)
            if dim == 3:
                g = kg[None, None, None, :] * self.ns + ecol_[:, :, :, None]
            else:
                g = kg[None, None, :] * self.ns + ecol_[:, :, 0][:, :, None]
            glob.append(g)
        glob_ = np.concatenate(glob, axis=0).reshape(E, -1)   # [e, local]

        return ecol_, xh_, yh_, glob_

    ecol = property(lambda self: self._arrays[0])
    xh = property(lambda self: self._arrays[1])
    yh = property(lambda self: self._arrays[2])
    glob = property(lambda self: self._arrays[3])

    # ------------------------------------------------------------------
    def surface_coords(self):
        """Physical (x, y) of each surface column (periodic: the first copy)."""
        x = np.zeros(self.ns)
        y = np.zeros(self.ns)
        # write in reverse element order so that the lowest element's value wins;
        # for periodic boxes this gives the wrapped column its x = 0 coordinate
        ec = self.ecol.reshape(-1)[::-1]
        x[ec] = self.xh.reshape(-1)[::-1]
        y[ec] = self.yh.reshape(-1)[::-1]
        return x, y

    def element_coords(self, eta, h):
        """Nodal (x, y, z) of every volume element, shape (E, n^dim) each.
        z = -h + sigma (eta + h) with uniform layers (Step 4.1, Sec. 3.1.2)."""
        dt_ = np.result_type(np.asarray(eta), np.asarray(h), np.float64)   # complex for the complex-step TLM
        eta = np.asarray(eta, dtype=dt_)
        h = np.asarray(h, dtype=dt_)
        xi = self.rule.xi
        xs, ys, zs = [], [], []
        for ez in range(self.nz):
            sigma = (ez + (1 + xi) / 2) / self.nz          # (n,) over local k
            if self.dim == 3:
                ec = self.ecol                             # (C, n, n)
                z = -h[ec][..., None] + sigma[None, None, None, :] * (eta[ec] + h[ec])[..., None]
                x = np.broadcast_to(self.xh[..., None], z.shape)
                y = np.broadcast_to(self.yh[..., None], z.shape)
            else:
                ec = self.ecol[:, :, 0]                    # (C, n)
                z = -h[ec][..., None] + sigma[None, None, :] * (eta[ec] + h[ec])[..., None]
                x = np.broadcast_to(self.xh[:, :, 0][..., None], z.shape)
                y = np.zeros(z.shape)
            xs.append(x.reshape(self.n_ecol, -1))
            ys.append(y.reshape(self.n_ecol, -1))
            zs.append(z.reshape(self.n_ecol, -1))
        return (np.concatenate(xs), np.concatenate(ys), np.concatenate(zs))

    def dof_counts(self):
        return self.N, self.ns
