"""Parity at the full sizes of the benchmark configurations, in the launch
configuration bench.py times (autotuned shapes, stored metric, p-multigrid,
graph-replayed steps): outputs the oracle can compute one at a time (operator
rows from the element matrices of the elements around a node; the vertical
velocity of a column from the GPU potential) and properties that hold at any
size (the oracle's residual of the GPU solve with its own matrix-free
operator)."""
import math

import numpy as np
import pytest
import torch

from oracle import mesh as omesh
from oracle import operator as oop
from oracle import solve as osolve
from paper_2506_09435_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def T(a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device=torch.device("cuda:0"))


def sampled_rows(om, op, x, y, rng, k=40):
    rows = rng.choice(om.N, size=k, replace=False)
    ref = np.array([op.row(int(i), x) for i in rows])
    scale = np.max(np.abs(y))
    return np.max(np.abs(y[rows] - ref)) / scale


def box_c2(fnpf, opts):
    d = W.periodic_box_3d()
    om = omesh.Mesh(3, d["nx"], d["ny"], d["nz"], d["p"], True, True, d["Lx"], d["Ly"])
    x, y = om.surface_coords()
    h = np.full(om.ns, d["h0"])
    eta, phis = W.airy_plus_spectrum_state(d, x, y, seed=2)
    gm = fnpf.Mesh(3, d["nx"], d["ny"], d["nz"], d["p"], True, True, h, Lx=d["Lx"], Ly=d["Ly"], g=d["g"],
                   opts=opts)
    return d, om, gm, h, eta, phis


def test_c2_full_size_operator_solve_and_w(fnpf):
    """32 x 32 x 2, p = 6 (479,232 DOF): operator rows, the solve's residual under
    the oracle's operator, and w at sampled columns."""
    opts = fnpf.default_opts(rtol=1e-10, precond=fnpf.FNPF_PMG)
    d, om, gm, h, eta, phis = box_c2(fnpf, opts)
    rng = np.random.default_rng(0)
    op = oop.Operator(om, eta, h, assemble=False)
    xv = rng.standard_normal(om.N)
    y = torch.empty(om.N, dtype=torch.float64, device="cuda:0")
    gm.apply(T(eta), T(xv), y)
    torch.cuda.synchronize()
    assert sampled_rows(om, op, xv, y.cpu().numpy(), rng) < 1e-12
    # solve (FP64, stored metric, p-multigrid): oracle residual of the GPU potential
    phi = torch.zeros(om.N, dtype=torch.float64, device="cuda:0")
    info = gm.laplace_solve(T(eta), T(phis), phi)
    assert info["status"] == 0 and info["rel_res"] <= 1e-10
    ph = phi.cpu().numpy()
    nI = om.n_interior
    b = -op.apply(np.concatenate([np.zeros(nI), phis]))[:nI]
    r = b - op.apply(np.concatenate([ph[:nI], np.zeros(om.ns)]))[:nI]
    assert np.linalg.norm(r) <= 2e-10 * np.linalg.norm(b)
    # vertical velocity of sampled columns from the GPU potential (oracle's general-inverse formula)
    w = torch.empty(om.ns, dtype=torch.float64, device="cuda:0")
    gm.dtn(T(eta), T(phis), w)
    w_ref = osolve.vertical_velocity(om, eta, h, ph)
    assert np.max(np.abs(w.cpu().numpy() - w_ref)) < 1e-9 * np.max(np.abs(w_ref))


def test_c2_full_size_mixed_matches_fp64(fnpf):
    """The benchmark's mixed-precision path on the same full-size tank: two RK4 steps
    agree with the FP64 path to 1e-8 relative (both graph-replayed after the first)."""
    outs = []
    for prec in (fnpf.FNPF_FP64, fnpf.FNPF_MIXED):
        opts = fnpf.default_opts(rtol=1e-10, precond=fnpf.FNPF_PMG, precision=prec)
        d, om, gm, h, eta, phis = box_c2(fnpf, opts)
        e, p = T(eta), T(phis)
        dt = W.period(d["k"], d["h0"], d["g"]) / 100
        for n in range(3):
            gm.rk4_step(e, p, n * dt, dt)
        torch.cuda.synchronize()
        outs.append((e.cpu().numpy(), p.cpu().numpy()))
    for a, b in zip(outs[0], outs[1]):
        assert np.linalg.norm(a - b) <= 1e-8 * np.linalg.norm(a)


def test_c3_bar_full_size_operator_rows(fnpf):
    """Submerged-bar flume 256 x 16 x 3, p = 5 (1,660,176 DOF, walls, variable depth)."""
    d = W.bar_flume()
    om = omesh.Mesh(3, d["nx"], d["ny"], d["nz"], d["p"], False, False, d["Lx"], d["Ly"])
    x, y = om.surface_coords()
    h = W.bar_depth(x)
    eta = 0.01 * np.cos(d["k"] * x) * (x < 20)
    gm = fnpf.Mesh(3, d["nx"], d["ny"], d["nz"], d["p"], False, False, h, Lx=d["Lx"], Ly=d["Ly"], g=d["g"])
    assert (gm.N, gm.ns) == (1660176, 103761)
    op = oop.Operator(om, eta, h, ops=[], assemble=False)
    rng = np.random.default_rng(1)
    xv = rng.standard_normal(om.N)
    yv = torch.empty(om.N, dtype=torch.float64, device="cuda:0")
    gm.apply(T(eta), T(xv), yv)
    yf = torch.empty(om.N, dtype=torch.float32, device="cuda:0")
    gm.apply_f32(T(eta).float(), T(xv).float(), yf)
    torch.cuda.synchronize()
    assert sampled_rows(om, op, xv, yv.cpu().numpy(), rng) < 1e-12
    assert sampled_rows(om, op, xv, yf.double().cpu().numpy(), rng) < 2e-6


def test_c4_cylinder_full_size_operator_rows(fnpf):
    """O-grid 64 x 24 x 3, p = 4 around the cylinder (isoparametric, 322,816 DOF)."""
    d = W.cylinder_case()
    box = omesh.Mesh(3, d["nx"], d["ny"], d["nz"], d["p"], True, False, d["Lx"], d["Ly"])
    th, s = box.surface_coords()
    X, Y = W.ogrid_map(th, s, a=d["a"], R=d["R"])
    om = omesh.Mesh(3, d["nx"], d["ny"], d["nz"], d["p"], True, False, X=X, Y=Y)
    h = np.full(om.ns, d["h0"])
    eta = 0.01 * np.cos(d["k"] * X)
    gm = fnpf.Mesh(3, d["nx"], d["ny"], d["nz"], d["p"], True, False, h, X=X, Y=Y, g=d["g"])
    assert (gm.N, gm.ns) == (322816, 24832)
    op = oop.Operator(om, eta, h, ops=[], assemble=False)
    rng = np.random.default_rng(2)
    xv = rng.standard_normal(om.N)
    yv = torch.empty(om.N, dtype=torch.float64, device="cuda:0")
    gm.apply(T(eta), T(xv), yv)
    torch.cuda.synchronize()
    assert sampled_rows(om, op, xv, yv.cpu().numpy(), rng) < 1e-12
