"""The prism leg of the step benchmark (bench.prism_leg) end to end on the
CPU: the library binding is replaced by the host harness of the prism step
(tests/emu, the kernels' own bodies run item by item) and CUDA events by a
stand-in, so that the leg's own logic -- mesh and zones, the timed steps, the
Jacobi comparison, the oracle child process and the error against it -- runs
as on the GPU, on a small flume."""
import sys
import types

import numpy as np
import pytest
import torch

import bench
from paper_2506_09435_gb300 import fnpf as F
from tests.emu import prism_emu as E


class _Event:
    def __init__(self, enable_timing=False):
        pass

    def record(self, stream=None):
        pass

    def elapsed_time(self, other):
        return 1.0


@pytest.fixture
def fake_binding(monkeypatch, tmp_path):
    hs = E.Harness(E.build(str(tmp_path)))

    class PrismMesh:
        def __init__(self, verts, tris, p, nz):
            self.em = hs.mesh(verts, tris, p, nz)
            self.N, self.ns = self.em.N, self.em.ns

        @staticmethod
        def default_opts(rtol=1e-10, g=9.81, precond=F.FNPF_JACOBI, precision=F.FNPF_FP64, projection=0):
            return E.opts(rtol=rtol, g=g, pmg=precond == F.FNPF_PMG, pc32=precision == F.FNPF_FP64_PC32,
                          mixed=precision == F.FNPF_MIXED, projection=projection)

        def set_relaxation(self, cr, gen, amp, kx, ky, omega, phase, ramp_time):
            self.em.set_relaxation(cr, gen, amp, kx, ky, omega, phase, ramp_time)

        def apply_stored(self, eta, h, x, y):
            y.copy_(torch.from_numpy(self.em.apply_stored(eta.numpy(), h.numpy(), x.numpy())))

        def apply(self, eta, h, x, y):
            self.apply_stored(eta, h, x, y)

        def diagonal(self, eta, h, d):
            d.copy_(torch.from_numpy(self.em.diagonal(eta.numpy(), h.numpy())))

        def step_adjoint(self, h, e, p, le, lp, oe, op, dt, lam_h=None, opts=None, t=0.0):
            st, a, b, c = self.em.step_adjoint(opts, h.numpy(), e.numpy(), p.numpy(), le.numpy(), lp.numpy(), dt, t=t)
            assert st == 0
            oe.copy_(torch.from_numpy(a))
            op.copy_(torch.from_numpy(b))
            lam_h.copy_(torch.from_numpy(c))

        def rk4_step(self, h, eta, phis, dt, opts, t=0.0):
            st, iters = self.em.rk4_step(opts, h.numpy(), eta.numpy(), phis.numpy(), dt, t=t)
            assert st == 0
            return [{"iters": i} for i in iters]

    fake = types.SimpleNamespace(PrismMesh=PrismMesh, prism_numbering=F.prism_numbering,
                                 FNPF_PMG=F.FNPF_PMG, FNPF_JACOBI=F.FNPF_JACOBI, FNPF_FP64=F.FNPF_FP64,
                                 FNPF_FP64_PC32=F.FNPF_FP64_PC32, FNPF_MIXED=F.FNPF_MIXED)
    import paper_2506_09435_gb300 as pkg
    monkeypatch.setattr(pkg, "fnpf", fake)
    monkeypatch.setattr(torch.cuda, "Event", _Event)
    monkeypatch.setattr(torch.cuda, "synchronize", lambda *a: None)
    monkeypatch.setattr(torch.cuda, "current_stream", lambda *a: None)
    yield
    monkeypatch.setattr(pkg, "fnpf", F)


def test_prism_leg_reports_throughput_iterations_and_oracle_error(fake_binding):
    args = types.SimpleNamespace(steps=2, rtol=1e-10, no_cpu_baseline=False)
    out = bench.prism_leg(torch.device("cpu"), args, None, size=(6, 2, 3, 2), sample=(4, 1, 2, 1, 2))
    assert out["finite"] and out["steps"] == 2 and out["dof"] > 0 and out["value"] > 0
    assert 0 < out["cg_iters_per_solve_mean"] < out["jacobi"]["cg_iters_per_solve_mean"]
    op = out["operator"]
    assert op["stored_metric"]["flops_executed"] > 0 and "us_per_application" in op["metric_per_application"], op
    assert out["adjoint"]["ratio"] > 0, out["adjoint"]
    mx = out["mixed"]
    assert mx["rel_l2_vs_fp64"]["eta"] <= 1e-8 and mx["rel_l2_vs_fp64"]["phis"] <= 1e-8, mx
    pc = out["fp64_pc32"]
    assert pc["rel_l2_vs_fp64"]["eta"] <= 1e-8 and pc["rel_l2_vs_fp64"]["phis"] <= 1e-8, pc
    assert out["cpu_baseline"]["kind"] == "oracle" and out["cpu_baseline"]["cores"] == 1
    err = out["rel_l2_vs_oracle"]
    assert err["eta"] <= 1e-10 and err["phis"] <= 1e-10, err
