"""The library's prism operator (fnpf_prism_apply: prisms over an unstructured
triangular surface mesh, Sec. 3.1.2) element by element against the oracle's
assembled matrix (oracle/prism.py), on jittered triangulations with curved
surface and bottom, p = 1..4, one and several layers; constants in the null
space; deterministic (two applications bitwise equal)."""
import numpy as np
import pytest
import torch

from oracle import prism as P
from paper_2506_09435_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("p", [1, 2, 3, 4])
@pytest.mark.parametrize("nz", [1, 3])
def test_prism_apply_matches_oracle(fnpf, p, nz):
    v, t = W.triangulated_box(3, 2, 1.3, 1.0)
    gm = fnpf.PrismMesh(v, t, p, nz)
    pm = P.PrismMesh(P.TriMesh(v, t, p), nz)
    assert gm.ns == pm.ns and gm.N == pm.N
    rng = np.random.default_rng(10 * p + nz)
    x_, y_ = pm.tm.xs, pm.tm.ys
    eta = 0.05 * np.cos(2.0 * x_) * np.sin(3.0 * y_)
    h = 0.6 - 0.1 * np.exp(-((x_ - 0.6) ** 2 + (y_ - 0.5) ** 2) / 0.05)
    xv = rng.standard_normal(pm.N)
    ref = pm.assemble(eta, h) @ xv
    dev = torch.device("cuda:0")
    T = lambda a: torch.tensor(a, dtype=torch.float64, device=dev)
    y1, y2 = torch.zeros(pm.N, dtype=torch.float64, device=dev), torch.zeros(pm.N, dtype=torch.float64, device=dev)
    gm.apply(T(eta), T(h), T(xv), y1)
    gm.apply(T(eta), T(h), T(xv), y2)
    ones = torch.zeros_like(y1)
    gm.apply(T(eta), T(h), torch.ones_like(y1), ones)
    torch.cuda.synchronize()
    y = y1.cpu().numpy()
    assert np.max(np.abs(y - ref)) <= 1e-12 * np.max(np.abs(ref))
    assert torch.equal(y1, y2)
    assert float(ones.abs().max()) <= 1e-12 * np.max(np.abs(ref))
