"""The checkpointed prism RK4 loop (autograd.prism_rk4_run) on the CPU: its
forward and backward run the prism step's kernel bodies through the host
harness (tests/emu) in place of the library binding, and the gradients of
J = sum(eta_N^2) + sum(phi_N) in eta0, phis0 and h equal the oracle's
complex-step derivatives; segments of 2 steps over 3 steps exercise the
checkpoint recomputation."""
import numpy as np
import pytest
import torch

from oracle import prism as P
from paper_2506_09435_gb300 import autograd as AG
from tests import prism_cases as C
from tests.emu import prism_emu as E


class _HarnessMesh:
    """The PrismMesh calls the loop makes, on torch CPU tensors."""

    def __init__(self, em):
        self.em = em

    def rk4_step(self, h, eta, phis, dt, opts, t=0.0):
        st, _ = self.em.rk4_step(opts, h.numpy(), eta.numpy(), phis.numpy(), dt, t=t)
        assert st == 0

    def step_adjoint(self, h, e, p, le, lp, oe, op, dt, lam_h=None, opts=None, t=0.0):
        st, a, b, c = self.em.step_adjoint(opts, h.numpy(), e.numpy(), p.numpy(), le.numpy(), lp.numpy(), dt, t=t)
        assert st == 0
        oe.copy_(torch.from_numpy(a))
        op.copy_(torch.from_numpy(b))
        lam_h.copy_(torch.from_numpy(c))


@pytest.fixture(scope="module")
def harness(tmp_path_factory):
    return E.Harness(E.build(str(tmp_path_factory.mktemp("prism_ag"))))


def test_checkpointed_gradients_match_oracle_complex_step(harness):
    p, nz = 2, 1
    v, t, pm = C.mesh(p, nz, nx=2, ny=1)
    eta0, h0, phis0 = C.fields(pm)
    o = E.opts(rtol=1e-13, mass_rtol=1e-14, g=C.G)
    mesh = _HarnessMesh(harness.mesh(v, t, p, nz))
    dt, nsteps = 0.02, 3
    e = torch.tensor(eta0, requires_grad=True)
    ph = torch.tensor(phis0, requires_grad=True)
    hh = torch.tensor(h0, requires_grad=True)
    eN, pN = AG.prism_rk4_run(mesh, e, ph, hh, 0.0, dt, nsteps, every=2, opts=o)
    (eN.pow(2).sum() + pN.sum()).backward()

    def J(de, dp, dh):
        x, y = eta0 + de, phis0 + dp
        for _ in range(nsteps):
            x, y = P.rk4_step(pm, h0 + dh, x, y, dt, C.G)
        return (x * x).sum() + y.sum()

    eps, z = 1e-30, np.zeros(pm.ns, dtype=complex)
    for grad, which in ((e.grad, 0), (ph.grad, 1), (hh.grad, 2)):
        ref = np.zeros(pm.ns)
        for c in range(pm.ns):
            d = [z.copy(), z.copy(), z.copy()]
            d[which][c] = 1j * eps
            ref[c] = J(*d).imag / eps
        assert C.rel(grad.numpy(), ref) <= 1e-9
