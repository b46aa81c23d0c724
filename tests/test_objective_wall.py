"""The cylinder-force objective of the differentiation form
(paper_2506_09435_gb300/objectives.py, torch operations) against the oracle's
functionals (oracle/wall.py) on the CPU: the values P and K of a curved,
moving-surface state, and their torch.autograd gradients with respect to the
volume potential, the elevation and the depth against the oracle's
complex-step derivatives."""
import math
from types import SimpleNamespace

import numpy as np
import pytest
import torch

from oracle import mesh as omesh
from oracle import wall
from paper_2506_09435_gb300 import workloads as W


def setup(p=3, nth=8, nr=2, nz=2, seed=0):
    box = omesh.Mesh(3, nth, nr, nz, p, periodic_x=True, periodic_y=False, Lx=2 * math.pi, Ly=1.0)
    th, s = box.surface_coords()
    X, Y = W.ogrid_map(th, s, a=1.0, R=3.0)
    m = omesh.Mesh(3, nth, nr, nz, p, periodic_x=True, periodic_y=False, X=X, Y=Y)
    rng = np.random.default_rng(seed)
    h = 1.0 + 0.1 * np.cos(X + 0.3) * np.exp(-(Y - 0.5) ** 2)
    eta = 0.05 * np.cos(X) + 0.02 * np.sin(2 * Y)
    phi = rng.standard_normal(m.N) * 0.1
    stand_in = SimpleNamespace(dim=3, nx=nth, ny=nr, nz=nz, p=p, periodic_x=True, periodic_y=False, ns=m.ns, N=m.N)
    return m, stand_in, X, Y, h, eta, phi


@pytest.mark.parametrize("p", [3, 5])
def test_objective_values_match_oracle(p):
    from paper_2506_09435_gb300.objectives import WallForce
    m, sm, X, Y, h, eta, phi = setup(p=p)
    wf = WallForce(sm, X, Y, Mz=p + 2, device=torch.device("cpu"))
    t = lambda a: torch.tensor(a, dtype=torch.float64)
    P, K = wf.evaluate(t(eta), t(h), t(phi))
    Pr, Kr = wall.wall_functionals(m, eta, h, phi, Mz=p + 2)
    assert abs(float(P) - Pr) <= 1e-12 * abs(Pr) and abs(float(K) - Kr) <= 1e-12 * abs(Kr)


def test_objective_gradients_match_oracle_complex_step():
    from paper_2506_09435_gb300.objectives import WallForce
    m, sm, X, Y, h, eta, phi = setup(p=3)
    wf = WallForce(sm, X, Y, Mz=5, device=torch.device("cpu"))
    te = torch.tensor(eta, dtype=torch.float64, requires_grad=True)
    th = torch.tensor(h, dtype=torch.float64, requires_grad=True)
    tp = torch.tensor(phi, dtype=torch.float64, requires_grad=True)
    P, K = wf.evaluate(te, th, tp)
    (P + 3.0 * K).backward()
    rng = np.random.default_rng(7)
    de, dh, dp = rng.standard_normal(m.ns), rng.standard_normal(m.ns), rng.standard_normal(m.N)
    eps = 1e-30
    Pc, Kc = wall.wall_functionals(m, eta + 1j * eps * de, h + 1j * eps * dh, phi + 1j * eps * dp, Mz=5)
    ref = np.imag(Pc + 3.0 * Kc) / eps
    got = te.grad.numpy() @ de + th.grad.numpy() @ dh + tp.grad.numpy() @ dp
    assert abs(got - ref) <= 1e-11 * abs(ref), (got, ref)
