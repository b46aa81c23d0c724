"""Batched groups of the ensemble: tanks of one order share every kernel
launch of the RK4 step (one launch over the concatenated grids, device-side
loops that run while any tank's loop runs, per-tank gates).  Each tank still
executes exactly the operations of its own step, so the batched ensemble
equals the tanks stepped one at a time bit for bit (with the same kernel
shapes), equals the oracle's RK4 steps, and launches far fewer kernels than
one branch of per-tank kernels per tank."""
import numpy as np
import pytest
import torch

from oracle import mesh as omesh
from oracle import surface as osurf
from paper_2506_09435_gb300 import workloads as W
from tests.pairs import rel_l2

pytestmark = pytest.mark.gpu

PREC = {"fp64": "FNPF_FP64", "mixed": "FNPF_MIXED", "pc32": "FNPF_FP64_PC32"}


def ragged_tanks():
    """Seven periodic tanks, three orders (p = 3, 3, 3, 4, 4, 5, 2), element
    counts 3..7 per direction (nx != ny), kh and steepness from the ensemble
    generator; the fourth p = 3 tank starts at rest, so its solves converge at
    once while the others iterate."""
    base = W.ensemble_tanks(n=7, seed=21, nmin=3, nmax=7, pmin=3, pmax=3)
    orders = [3, 3, 3, 4, 4, 5, 2]
    out = []
    for d, p in zip(base, orders):
        e = W.periodic_box_3d(nx=d["nx"], ny=d["ny"], nz=2, p=p, kh=d["k"] * d["h0"])
        e.update(steepness=d["steepness"], seed=d["seed"])
        out.append(e)
    out[2]["rest"] = True
    return out


def build(fnpf, tanks, opts, shapes):
    dev = torch.device("cuda:0")
    meshes, etas, phiss, dts = [], [], [], []
    for d in tanks:
        ncx, ncy = d["p"] * d["nx"], d["p"] * d["ny"]
        m = fnpf.Mesh(3, d["nx"], d["ny"], 2, d["p"], True, True, np.full(ncx * ncy, d["h0"]), Lx=d["Lx"],
                      Ly=d["Ly"], g=d["g"], opts=opts)
        if shapes is not None:
            m.set_shapes(*shapes)
        x, y = m.surface_coords()
        e0, p0 = W.airy_plus_spectrum_state(d, x, y, seed=d["seed"], steepness=d["steepness"])
        if d.get("rest"):
            e0, p0 = np.zeros_like(e0), np.zeros_like(p0)
        meshes.append(m)
        etas.append(torch.tensor(e0, dtype=torch.float64, device=dev))
        phiss.append(torch.tensor(p0, dtype=torch.float64, device=dev))
        dts.append(W.period(d["k"], d["h0"], d["g"]) / 100)
    return meshes, etas, phiss, dts


@pytest.mark.parametrize("prec", ["fp64", "mixed", "pc32"])
def test_batched_groups_equal_tanks_stepped_one_at_a_time(fnpf, prec):
    tanks = ragged_tanks()
    o = fnpf.default_opts(rtol=1e-10, precond=fnpf.FNPF_PMG, precision=getattr(fnpf, PREC[prec]))
    meshes, etas, phiss, dts = build(fnpf, tanks, o, (1, 1))
    ens = fnpf.Ensemble(meshes)
    infos = []
    for k in range(4):
        infos.append(ens.rk4_step(etas, phiss, [k * dt for dt in dts], dts, info=True))
    torch.cuda.synchronize()
    st = ens.stats()
    assert st["groups"] == 2 and st["batched_tanks"] == 5, st      # p = 3 (3 tanks), p = 4 (2); p = 5, 2 alone
    ref_m, ref_e, ref_p, _ = build(fnpf, tanks, o, (1, 1))
    ref_infos = []
    for k in range(4):
        ref_infos.append([m.rk4_step(e, p, k * dt, dt, info=True) for m, e, p, dt in zip(ref_m, ref_e, ref_p, dts)])
    torch.cuda.synchronize()
    for i, (a, b, c, d) in enumerate(zip(etas, ref_e, phiss, ref_p)):
        assert torch.equal(a, b) and torch.equal(c, d), i
    # the same iteration counts per tank and stage (batched steps 2..4)
    for k in range(1, 4):
        for i in range(len(tanks)):
            for s in range(4):
                assert infos[k][4 * i + s]["iters"] == ref_infos[k][i][s]["iters"], (k, i, s)
    assert all(v == 0 for v in etas[2].cpu().numpy()) and all(v == 0 for v in phiss[2].cpu().numpy())


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-10), ("mixed", 1e-8), ("pc32", 1e-10)])
def test_batched_groups_match_oracle(fnpf, prec, tol):
    tanks = ragged_tanks()
    o = fnpf.default_opts(rtol=1e-13, precond=fnpf.FNPF_PMG, precision=getattr(fnpf, PREC[prec]), max_iter=50000)
    meshes, etas, phiss, dts = build(fnpf, tanks, o, None)
    init = [(e.cpu().numpy(), p.cpu().numpy()) for e, p in zip(etas, phiss)]
    ens = fnpf.Ensemble(meshes)
    for k in range(3):
        ens.rk4_step(etas, phiss, [k * dt for dt in dts], dts)
    torch.cuda.synchronize()
    assert ens.stats()["batched_tanks"] == 5
    for i, d in enumerate(tanks):
        om = omesh.Mesh(3, d["nx"], d["ny"], 2, d["p"], True, True, d["Lx"], d["Ly"])
        h = np.full(om.ns, d["h0"])
        e_r, p_r = init[i]
        for _ in range(3):
            e_r, p_r = osurf.rk4_step(om, h, e_r, p_r, dts[i], d["g"])
        if d.get("rest"):
            assert not np.any(etas[i].cpu().numpy()) and not np.any(phiss[i].cpu().numpy())
            continue
        assert rel_l2(etas[i].cpu().numpy(), e_r) < tol, (i, d["p"])
        assert rel_l2(phiss[i].cpu().numpy(), p_r) < tol, (i, d["p"])


def test_group_limits(fnpf):
    """Groups of at most max_tanks tanks and max_dof degrees of freedom, filled
    in increasing size; a group of one runs on its own; the results stay
    bitwise those of the tanks stepped one at a time."""
    tanks = [t for t in ragged_tanks() if t["p"] == 3] * 2           # six p = 3 tanks (two at rest)
    o = fnpf.default_opts(rtol=1e-10, precond=fnpf.FNPF_PMG, precision=fnpf.FNPF_FP64)
    meshes, etas, phiss, dts = build(fnpf, tanks, o, (1, 1))
    sizes = sorted(m.N for m in meshes)
    ens = fnpf.Ensemble(meshes)
    ens.set_batching(True, max_tanks=4, max_dof=sizes[0] + sizes[1] + sizes[2])
    for k in range(3):
        ens.rk4_step(etas, phiss, [k * dt for dt in dts], dts)
    torch.cuda.synchronize()
    st = ens.stats()
    assert 1 <= st["groups"] <= 3 and st["batched_tanks"] <= 6, st
    ref_m, ref_e, ref_p, _ = build(fnpf, tanks, o, (1, 1))
    for k in range(3):
        for m, e, p, dt in zip(ref_m, ref_e, ref_p, dts):
            m.rk4_step(e, p, k * dt, dt)
    torch.cuda.synchronize()
    for a, b in zip(etas + phiss, ref_e + ref_p):
        assert torch.equal(a, b)
    with pytest.raises(fnpf.FnpfError):
        ens.set_batching(True, max_tanks=33)


def test_batching_cuts_kernel_launches(fnpf):
    """The same ensemble step with and without batched groups: equal states,
    and fewer kernels for the batched step (two groups of four tanks: a group
    runs each loop as long as its slowest tank, so the cut is below 4x)."""
    tanks = [t for t in ragged_tanks() if not t.get("rest")]
    tanks = tanks[:2] + tanks[:2] + tanks[2:4] + tanks[2:4]      # 4 tanks of p = 3, 4 of p = 4
    o = fnpf.default_opts(rtol=1e-10, precond=fnpf.FNPF_PMG, precision=fnpf.FNPF_MIXED)
    out, kernels = [], []
    for batching in (False, True):
        meshes, etas, phiss, dts = build(fnpf, tanks, o, (1, 1))
        ens = fnpf.Ensemble(meshes)
        ens.set_batching(batching)
        for k in range(3):
            ens.rk4_step(etas, phiss, [k * dt for dt in dts], dts)
        torch.cuda.synchronize()
        kernels.append(ens.stats()["kernels"])
        out.append([t.cpu().numpy() for t in etas + phiss])
    for a, b in zip(*out):
        assert np.array_equal(a, b)
    assert kernels[1] * 2 < kernels[0], kernels


def test_same_mesh_twice_is_rejected(fnpf):
    tanks = ragged_tanks()[:1]
    o = fnpf.default_opts(rtol=1e-10)
    meshes, _, _, _ = build(fnpf, tanks, o, None)
    with pytest.raises(fnpf.FnpfError):
        fnpf.Ensemble([meshes[0], meshes[0]])


def relax_flumes(fnpf, opts):
    """Three walled flumes of one order over the bar bathymetry (different
    lengths, so different element counts), generation and absorption zones."""
    out = []
    for nx, Lx in ((8, 8.0), (10, 10.0), (12, 12.0)):
        d = W.bar_flume(nx=nx, ny=2, nz=2, p=3, Lx=Lx)
        d["zone"] = Lx / 4
        gm = fnpf.Mesh(3, nx, 2, 2, 3, False, False, np.full((3 * nx + 1) * 7, d["h0"]), Lx=Lx, Ly=d["Ly"],
                       g=d["g"], opts=opts)
        x, _ = gm.surface_coords()
        h = W.bar_depth(x * 38.0 / Lx)
        gm = fnpf.Mesh(3, nx, 2, 2, 3, False, False, h, Lx=Lx, Ly=d["Ly"], g=d["g"], opts=opts)
        gm.set_shapes(1, 1)
        cr, gen = W.flume_zones(d, x)
        gm.set_relaxation(cr, gen, **W.flume_wave(d))
        out.append((d, gm))
    return out


def test_batched_relaxation_flumes_equal_one_at_a_time(fnpf):
    """The relaxation blend of the last stage reads each tank's own step time
    on the device (written by the host before every graph launch): a batched
    group of flumes started at different times equals the flumes stepped one at
    a time, bit for bit, and the generation zones have started their waves."""
    o = fnpf.default_opts(rtol=1e-10, precond=fnpf.FNPF_PMG)
    dev = torch.device("cuda:0")
    runs = []
    for batched in (True, False):
        fl = relax_flumes(fnpf, o)
        etas = [torch.zeros(m.ns, dtype=torch.float64, device=dev) for _, m in fl]
        phiss = [torch.zeros_like(e) for e in etas]
        dts = [d["T"] / 50 for d, _ in fl]
        t0 = [0.0, 0.3, 0.7]
        if batched:
            ens = fnpf.Ensemble([m for _, m in fl])
            for k in range(5):
                ens.rk4_step(etas, phiss, [a + k * dt for a, dt in zip(t0, dts)], dts)
            assert ens.stats()["batched_tanks"] == 3
        else:
            for k in range(5):
                for (d, m), e, p, a, dt in zip(fl, etas, phiss, t0, dts):
                    m.rk4_step(e, p, a + k * dt, dt)
        torch.cuda.synchronize()
        runs.append([t.cpu().numpy() for t in etas + phiss])
    for a, b in zip(*runs):
        assert np.array_equal(a, b)
    assert all(np.max(np.abs(a)) > 0 for a in runs[0][:3])


def test_failing_tank_in_a_batched_group(fnpf):
    """A tank of a batched group whose state folds (eta + h <= 0) reports
    EDIVERGED for the ensemble step, named by index; the other tanks of its
    group still take exactly the step they take on their own."""
    tanks = [t for t in ragged_tanks() if t["p"] == 3 and not t.get("rest")] * 2   # four p = 3 tanks
    o = fnpf.default_opts(rtol=1e-10, precond=fnpf.FNPF_PMG)
    meshes, etas, phiss, dts = build(fnpf, tanks, o, (1, 1))
    ref_m, ref_e, ref_p, _ = build(fnpf, tanks, o, (1, 1))
    ens = fnpf.Ensemble(meshes)
    for k in range(2):
        ens.rk4_step(etas, phiss, [k * dt for dt in dts], dts)
        for m, e, p, dt in zip(ref_m, ref_e, ref_p, dts):
            m.rk4_step(e, p, k * dt, dt)
    assert ens.stats()["batched_tanks"] == 4
    etas[2].fill_(-10.0)                         # folded: eta + h < 0 everywhere
    ref_e[2].fill_(-10.0)
    with pytest.raises(fnpf.FnpfError, match="tank 2"):
        ens.rk4_step(etas, phiss, [2 * dt for dt in dts], dts)
    for i in (0, 1, 3):
        ref_m[i].rk4_step(ref_e[i], ref_p[i], 2 * dts[i], dts[i])
    torch.cuda.synchronize()
    for i in (0, 1, 3):
        assert torch.equal(etas[i], ref_e[i]) and torch.equal(phiss[i], ref_p[i]), i
