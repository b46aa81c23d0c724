"""Captured RK4-step graphs (device-side CG loops as conditional WHILE nodes)
and the batched ensemble: both run exactly the kernels of the host-driven path,
so results are bitwise identical; the ensemble advances tanks of different
sizes and orders in one launch and matches stepping them one at a time."""
import numpy as np
import pytest
import torch

from oracle import surface as osurf
from paper_2506_09435_gb300 import workloads as W
from tests.pairs import Case, rel_l2

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("prec,pre", [("fp64", "pmg"), ("fp64", "jacobi"), ("mixed", "pmg"), ("mixed", "jacobi")])
def test_step_graph_bitwise_equals_host_driven(fnpf, prec, pre):
    shape = (3, 5, 4, 2, 4, True, False)
    out = []
    for graphs in (0, 1):
        o = fnpf.default_opts(rtol=1e-11, use_graphs=graphs,
                              precision=fnpf.FNPF_MIXED if prec == "mixed" else fnpf.FNPF_FP64,
                              precond=fnpf.FNPF_PMG if pre == "pmg" else fnpf.FNPF_JACOBI)
        c = Case(fnpf, *shape, opts=o)
        c.gm.set_shapes(4, 4)   # the same kernels on both meshes (the autotuner could pick different ones)
        eta, phis = c.t(c.eta), c.t(c.phis)
        infos = [c.gm.rk4_step(eta, phis, 0.01 * k, 0.01, info=True) for k in range(4)]
        torch.cuda.synchronize()
        out.append((eta.cpu().numpy(), phis.cpu().numpy(), infos))
    assert np.array_equal(out[0][0], out[1][0]) and np.array_equal(out[0][1], out[1][1])
    for a, b in zip(out[0][2], out[1][2]):
        assert [s["iters"] for s in a] == [s["iters"] for s in b]
        assert all(s["status"] == 0 for s in b)


def test_step_graph_with_relaxation_matches_oracle(fnpf):
    d = W.bar_flume(nx=12, ny=2, nz=2, p=3, Lx=12.0)
    d["zone"] = 3.0
    from oracle import mesh as omesh
    om = omesh.Mesh(3, 12, 2, 2, 3, periodic_x=False, periodic_y=False, Lx=12.0, Ly=d["Ly"])
    x, _ = om.surface_coords()
    h = W.bar_depth(x * 38.0 / 12.0)
    gm = fnpf.Mesh(3, 12, 2, 2, 3, False, False, h, Lx=12.0, Ly=d["Ly"], g=d["g"],
                   opts=fnpf.default_opts(rtol=1e-13, precond=fnpf.FNPF_PMG))
    cr, gen = W.flume_zones(d, x)
    wave = W.flume_wave(d)
    gm.set_relaxation(cr, gen, **wave)
    dt = d["T"] / 100
    eta_r, phi_r = np.zeros(om.ns), np.zeros(om.ns)
    dev = torch.device("cuda:0")
    eta = torch.zeros(om.ns, dtype=torch.float64, device=dev)
    phis = torch.zeros_like(eta)
    for n in range(5):
        eta_r, phi_r = osurf.relaxation_step(om, h, eta_r, phi_r, n * dt, dt, d["g"], cr, gen, wave)
        gm.rk4_step(eta, phis, n * dt, dt)          # steps 2..5 replay the captured graph
    torch.cuda.synchronize()
    assert rel_l2(eta.cpu().numpy(), eta_r) < 1e-10
    assert rel_l2(phis.cpu().numpy(), phi_r) < 1e-10


def test_step_graph_reports_iteration_cap(fnpf):
    c = Case(fnpf, 3, 4, 3, 2, 4, True, True, opts=fnpf.default_opts(rtol=1e-12, max_iter=3))
    eta, phis = c.t(c.eta), c.t(c.phis)
    st = c.gm.rk4_step(eta, phis, 0.0, 0.01, check=False)
    assert st == fnpf.FNPF_ENOCONV
    c.gm.set_opts(fnpf.default_opts(rtol=1e-12))
    c.gm.rk4_step(eta, phis, 0.0, 0.01)                  # host-driven warm-up after the failure
    c.gm.set_opts(fnpf.default_opts(rtol=1e-12, max_iter=3))
    st = c.gm.rk4_step(eta, phis, 0.01, 0.01, check=False)  # captured graph, device-side cap
    assert st == fnpf.FNPF_ENOCONV


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_ensemble_matches_tanks_stepped_one_at_a_time(fnpf, prec):
    tanks = W.ensemble_tanks(n=5, seed=7, nmin=3, nmax=7, pmin=2, pmax=6)
    dev = torch.device("cuda:0")
    o = fnpf.default_opts(rtol=1e-10, precond=fnpf.FNPF_PMG,
                          precision=fnpf.FNPF_MIXED if prec == "mixed" else fnpf.FNPF_FP64)

    def setup():
        meshes, etas, phiss, dts = [], [], [], []
        for d in tanks:
            ncx = d["p"] * d["nx"]
            ncy = d["p"] * d["ny"]
            m = fnpf.Mesh(3, d["nx"], d["ny"], 2, d["p"], True, True, np.full(ncx * ncy, d["h0"]), Lx=d["Lx"],
                          Ly=d["Ly"], g=d["g"], opts=o)
            m.set_shapes(5, 5)   # the same kernels in both runs
            x, y = m.surface_coords()
            e0, p0 = W.airy_plus_spectrum_state(d, x, y, seed=d["seed"], steepness=d["steepness"])
            meshes.append(m)
            etas.append(torch.tensor(e0, dtype=torch.float64, device=dev))
            phiss.append(torch.tensor(p0, dtype=torch.float64, device=dev))
            dts.append(W.period(d["k"], d["h0"], d["g"]) / 100)
        return meshes, etas, phiss, dts

    meshes, etas, phiss, dts = setup()
    ens = fnpf.Ensemble(meshes)
    for k in range(3):
        ens.rk4_step(etas, phiss, [k * dt for dt in dts], dts)
    torch.cuda.synchronize()
    ref_m, ref_e, ref_p, _ = setup()
    for k in range(3):
        for m, e, p, dt in zip(ref_m, ref_e, ref_p, dts):
            m.rk4_step(e, p, k * dt, dt)
    torch.cuda.synchronize()
    for a, b in zip(etas + phiss, ref_e + ref_p):
        assert torch.equal(a, b)
