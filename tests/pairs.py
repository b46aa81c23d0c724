"""Builds an oracle mesh and a GPU mesh from one descriptor, with the same
seeded inputs on both sides (inputs come from the oracle's coordinates and
the workloads module, never from the CUDA path)."""
import math

import numpy as np

from oracle import mesh as omesh


class Case:
    def __init__(self, fnpf, dim, nx, ny, nz, p, px=True, py=True, Lx=1.0, Ly=1.0, h0=0.4, amp=0.03,
                 hvar=0.1, seed=0, opts=None, g=9.81):
        import torch
        self.dim, self.p = dim, p
        self.om = omesh.Mesh(dim, nx, ny, nz, p, periodic_x=px, periodic_y=py, Lx=Lx, Ly=Ly)
        x, y = self.om.surface_coords()
        self.x, self.y = x, y
        kx, ky = 2 * math.pi / Lx, (2 * math.pi / Ly if dim == 3 else 0.0)
        self.h = h0 * (1 + hvar * np.sin(kx * x + 0.3) * np.cos(ky * y))
        self.eta = amp * h0 * np.cos(kx * x + 0.1) * np.cos(ky * y + 0.2) \
            + 0.2 * amp * h0 * np.sin(2 * kx * x - 0.4)
        self.phis = 0.1 * np.sin(kx * x) * np.cos(ky * y) + 0.02 * np.cos(2 * kx * x + ky * y)
        self.gm = fnpf.Mesh(dim, nx, ny, nz, p, px, py, self.h, Lx=Lx, Ly=Ly, g=g, opts=opts)
        assert (self.gm.N, self.gm.ns) == (self.om.N, self.om.ns)
        gx, gy = self.gm.surface_coords()
        assert np.max(np.abs(gx - x)) < 1e-13 and np.max(np.abs(gy - y)) < 1e-13
        self.rng = np.random.default_rng(seed)
        self.dev = torch.device("cuda:0")

    def t(self, a):
        import torch
        return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device=self.dev)


def rel_l2(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(np.asarray(b)), 1e-300))


def rel_max(a, b):
    return float(np.max(np.abs(np.asarray(a) - np.asarray(b))) / max(np.max(np.abs(np.asarray(b))), 1e-300))
