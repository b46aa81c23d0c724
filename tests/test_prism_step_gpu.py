"""The prism solve, w, projected free-surface conditions and RK4 step on the
GPU (fnpf_prism_diagonal, fnpf_prism_apply_stored, fnpf_prism_laplace_solve,
fnpf_prism_dtn, fnpf_prism_rhs, fnpf_prism_rk4_step; Sec. 3.1.2 mesh, Sec. 3.4
Steps 4.1-4.6, Sec. 3.2 ERK4) element by element against the prism oracle
(oracle/prism.py) on the seeded inputs of tests/prism_cases.py; the operator
with the stored metric also against the library's on-the-fly prism operator."""
import numpy as np
import pytest
import torch

from oracle import prism as P
from tests import prism_cases as C

pytestmark = pytest.mark.gpu

DEV = torch.device("cuda:0")


def T(a):
    return torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device=DEV)


def opts(fnpf, rtol=1e-13, max_iter=20000, linear=False, pmg=False, pc32=False):
    return fnpf.PrismMesh.default_opts(rtol=rtol, max_iter=max_iter, mass_rtol=1e-13, g=C.G,
                                       model=fnpf.FNPF_LINEAR if linear else fnpf.FNPF_NONLINEAR,
                                       precond=fnpf.FNPF_PMG if (pmg or pc32) else fnpf.FNPF_JACOBI,
                                       precision=fnpf.FNPF_FP64_PC32 if pc32 else fnpf.FNPF_FP64)


@pytest.mark.parametrize("p", [1, 2, 3, 4])
@pytest.mark.parametrize("nz", [1, 3])
def test_stored_operator_and_diagonal_match_oracle(fnpf, p, nz):
    v, t, pm = C.mesh(p, nz)
    gm = fnpf.PrismMesh(v, t, p, nz)
    eta, h, _ = C.fields(pm)
    A = pm.assemble(eta, h)
    x = np.random.default_rng(100 + 10 * p + nz).standard_normal(pm.N)
    ref = A @ x
    ys, yf, d = (torch.zeros(pm.N, dtype=torch.float64, device=DEV) for _ in range(3))
    gm.apply_stored(T(eta), T(h), T(x), ys)
    gm.apply(T(eta), T(h), T(x), yf)
    gm.diagonal(T(eta), T(h), d)
    torch.cuda.synchronize()
    ys, yf, d = ys.cpu().numpy(), yf.cpu().numpy(), d.cpu().numpy()
    assert np.max(np.abs(ys - ref)) <= 1e-12 * np.max(np.abs(ref))
    assert np.max(np.abs(ys - yf)) <= 1e-12 * np.max(np.abs(ref))
    assert np.max(np.abs(d - A.diagonal())) <= 1e-13 * np.max(np.abs(A.diagonal()))


@pytest.mark.parametrize("p", [1, 2, 3, 4])
def test_laplace_solve_matches_oracle(fnpf, p):
    nz = 2
    v, t, pm = C.mesh(p, nz)
    gm = fnpf.PrismMesh(v, t, p, nz)
    eta, h, phis = C.fields(pm)
    phi = torch.zeros(pm.N, dtype=torch.float64, device=DEV)
    info = gm.laplace_solve(T(eta), T(h), T(phis), phi, opts(fnpf))
    assert info["status"] == 0 and info["iters"] > 0 and info["rel_res"] <= 1e-13
    ref = P.laplace_solve(pm, eta, h, phis)
    out = phi.cpu().numpy()
    assert C.rel(out, ref) <= 1e-10
    assert np.array_equal(out[pm.N - pm.ns:], phis)
    info = gm.laplace_solve(T(eta), T(h), T(phis), phi, opts(fnpf, rtol=1e-10))
    assert info["iters"] == 0 and C.rel(phi.cpu().numpy(), ref) <= 1e-10


def test_solve_special_cases(fnpf):
    p, nz = 3, 2
    v, t, pm = C.mesh(p, nz)
    gm = fnpf.PrismMesh(v, t, p, nz)
    eta, h, phis = C.fields(pm)
    phi = T(np.random.default_rng(1).standard_normal(pm.N))
    gm.laplace_solve(T(eta), T(h), T(np.full(pm.ns, 0.3)), phi, opts(fnpf))
    assert float((phi - 0.3).abs().max()) <= 1e-12
    phi = T(np.random.default_rng(2).standard_normal(pm.N))
    info = gm.laplace_solve(T(eta), T(h), T(np.zeros(pm.ns)), phi, opts(fnpf))
    assert info["iters"] == 0 and not bool(phi.any())
    with pytest.raises(fnpf.FnpfError) as e:
        gm.laplace_solve(T(eta), T(h), T(phis), torch.zeros(pm.N, dtype=torch.float64, device=DEV),
                         opts(fnpf, max_iter=2))
    assert e.value.status == fnpf.FNPF_ENOCONV
    e0, p0 = T(eta), T(phis)
    with pytest.raises(fnpf.FnpfError):
        gm.rk4_step(T(h), e0, p0, 0.01, opts(fnpf, max_iter=2))
    assert np.array_equal(e0.cpu().numpy(), eta) and np.array_equal(p0.cpu().numpy(), phis)


@pytest.mark.parametrize("linear", [False, True])
@pytest.mark.parametrize("p", [2, 3, 4])
def test_dtn_and_projected_conditions_match_oracle(fnpf, p, linear):
    nz = 2
    v, t, pm = C.mesh(p, nz)
    gm = fnpf.PrismMesh(v, t, p, nz)
    eta, h, phis = C.fields(pm)
    geo = np.zeros_like(eta) if linear else eta
    w = torch.zeros(pm.ns, dtype=torch.float64, device=DEV)
    gm.dtn(T(geo), T(h), T(phis), w, opts(fnpf, linear=linear))
    assert C.rel(w.cpu().numpy(), P.w_recovery(pm, geo, h, P.laplace_solve(pm, geo, h, phis))) <= 1e-10
    ke, kp = (torch.zeros(pm.ns, dtype=torch.float64, device=DEV) for _ in range(2))
    gm.rhs(T(eta), T(h), T(phis), ke, kp, opts(fnpf, linear=linear))
    ko = P.rhs(pm, h, eta, phis, C.G, linear=linear)
    assert C.rel(ke.cpu().numpy(), ko[0]) <= 1e-10 and C.rel(kp.cpu().numpy(), ko[1]) <= 1e-10


@pytest.mark.parametrize("linear", [False, True])
@pytest.mark.parametrize("p", [2, 4])
def test_rk4_steps_match_oracle(fnpf, p, linear):
    nz = 2
    v, t, pm = C.mesh(p, nz, nx=4, ny=3, seed=11)
    gm = fnpf.PrismMesh(v, t, p, nz)
    eta, h, phis = C.standing_wave(pm)
    e1, p1, hd = T(eta), T(phis), T(h)
    eo, po = eta.copy(), phis.copy()
    dt = 0.02
    for _ in range(3):
        infos = gm.rk4_step(hd, e1, p1, dt, opts(fnpf, linear=linear))
        assert all(i["status"] == 0 for i in infos) and max(i["iters"] for i in infos) > 0
        eo, po = P.rk4_step(pm, h, eo, po, dt, C.G, linear=linear)
    assert C.rel(e1.cpu().numpy(), eo) <= 1e-10 and C.rel(p1.cpu().numpy(), po) <= 1e-10


@pytest.mark.parametrize("p, alpha, order, cutoff", [(3, 2.0, 2, 0), (4, 36.0, 4, 1), (6, 1.0, 8, 3)])
def test_modal_filter_matches_oracle(fnpf, p, alpha, order, cutoff):
    v, t, pm = C.mesh(p, 1)
    gm = fnpf.PrismMesh(v, t, p, 1)
    f = np.random.default_rng(p).standard_normal(pm.ns)
    gm.set_filter(alpha, order, cutoff)
    fd = T(f)
    gm.filter_apply(fd)
    ref = P.apply_filter(pm.tm, f, alpha, order, cutoff)
    assert np.max(np.abs(fd.cpu().numpy() - ref)) <= 1e-12 * np.max(np.abs(f))
    gm.set_filter(0.0)
    with pytest.raises(fnpf.FnpfError) as e:
        gm.filter_apply(fd)
    assert e.value.status == fnpf.FNPF_EINVAL


@pytest.mark.parametrize("p", [3, 4])
def test_filtered_rk4_steps_match_oracle(fnpf, p):
    nz = 2
    v, t, pm = C.mesh(p, nz, nx=4, ny=3, seed=11)
    gm = fnpf.PrismMesh(v, t, p, nz)
    eta, h, _ = C.standing_wave(pm)
    phis = C.fields(pm)[2]
    gm.set_filter(4.0, 2, 1)
    e1, p1, hd = T(eta), T(phis), T(h)
    eo, po = eta.copy(), phis.copy()
    for _ in range(2):
        gm.rk4_step(hd, e1, p1, 0.02, opts(fnpf))
        eo, po = P.rk4_step(pm, h, eo, po, 0.02, C.G)
        eo, po = P.apply_filter(pm.tm, eo, 4.0, 2, 1), P.apply_filter(pm.tm, po, 4.0, 2, 1)
    assert C.rel(e1.cpu().numpy(), eo) <= 1e-10 and C.rel(p1.cpu().numpy(), po) <= 1e-10


@pytest.mark.parametrize("p, nz, nx, ny", [(2, 2, 3, 2), (4, 2, 6, 4), (5, 3, 4, 3)])
def test_pmg_solve_matches_oracle_in_fewer_iterations(fnpf, p, nz, nx, ny):
    v, t, pm = C.mesh(p, nz, nx=nx, ny=ny)
    gm = fnpf.PrismMesh(v, t, p, nz)
    eta, h, phis = C.fields(pm)
    phi_j = torch.zeros(pm.N, dtype=torch.float64, device=DEV)
    phi_m = torch.zeros(pm.N, dtype=torch.float64, device=DEV)
    info_j = gm.laplace_solve(T(eta), T(h), T(phis), phi_j, opts(fnpf))
    info_m = gm.laplace_solve(T(eta), T(h), T(phis), phi_m, opts(fnpf, pmg=True))
    assert info_m["status"] == 0 and info_m["rel_res"] <= 1e-13
    assert C.rel(phi_m.cpu().numpy(), P.laplace_solve(pm, eta, h, phis)) <= 1e-10
    assert info_m["iters"] * 3 <= info_j["iters"]


def test_vcycle_is_symmetric_positive_definite(fnpf):
    p, nz = 4, 2
    v, t, pm = C.mesh(p, nz, nx=3, ny=2)
    gm = fnpf.PrismMesh(v, t, p, nz)
    eta, h, _ = C.fields(pm)
    NI = pm.N - pm.ns
    rng = np.random.default_rng(5)
    u, w = rng.standard_normal(pm.N), rng.standard_normal(pm.N)
    u[NI:] = 0
    w[NI:] = 0
    Mu, Mw = (torch.zeros(pm.N, dtype=torch.float64, device=DEV) for _ in range(2))
    gm.precond_apply(T(eta), T(h), T(u), Mu, opts(fnpf, pmg=True))
    gm.precond_apply(T(eta), T(h), T(w), Mw, opts(fnpf, pmg=True))
    Mu, Mw = Mu.cpu().numpy(), Mw.cpu().numpy()
    assert not Mu[NI:].any()
    assert abs(w @ Mu - u @ Mw) <= 1e-12 * np.linalg.norm(u) * np.linalg.norm(Mw)
    assert u @ Mu > 0 and w @ Mw > 0


def test_pmg_rk4_steps_match_oracle(fnpf):
    p, nz = 4, 2
    v, t, pm = C.mesh(p, nz, nx=4, ny=3, seed=11)
    gm = fnpf.PrismMesh(v, t, p, nz)
    eta, h, phis = C.standing_wave(pm)
    e1, p1, hd = T(eta), T(phis), T(h)
    eo, po = eta.copy(), phis.copy()
    for _ in range(3):
        gm.rk4_step(hd, e1, p1, 0.02, opts(fnpf, pmg=True))
        eo, po = P.rk4_step(pm, h, eo, po, 0.02, C.G)
    assert C.rel(e1.cpu().numpy(), eo) <= 1e-10 and C.rel(p1.cpu().numpy(), po) <= 1e-10


@pytest.mark.parametrize("p, filt", [(2, None), (3, (4.0, 2, 1))])
def test_relaxation_zones_match_oracle(fnpf, p, filt):
    nz = 2
    v, t, pm, h, cr, gen, wave = C.flume(p, nz)
    gm = fnpf.PrismMesh(v, t, p, nz)
    gm.set_relaxation(cr, gen, wave["amp"], wave["kx"], wave["ky"], wave["omega"], wave["phase"], wave["ramp_time"])
    if filt:
        gm.set_filter(*filt)
    e1, p1, hd = T(np.zeros(pm.ns)), T(np.zeros(pm.ns)), T(h)
    eo, po = np.zeros(pm.ns), np.zeros(pm.ns)
    t0, dt = 4.0, 0.025
    for k in range(3):
        gm.rk4_step(hd, e1, p1, dt, opts(fnpf), t=t0 + k * dt)
        eo, po = P.relaxation_step(pm, h, eo, po, t0 + k * dt, dt, C.G, cr, gen, wave, filt=filt)
    assert C.rel(e1.cpu().numpy(), eo) <= 1e-10 and C.rel(p1.cpu().numpy(), po) <= 1e-10
    gm.set_relaxation(None, None, 0, 0, 0, 0, 0, 0)


@pytest.mark.parametrize("linear", [False, True])
def test_invariants_match_oracle(fnpf, linear):
    p, nz = 3, 2
    v, t, pm = C.mesh(p, nz)
    gm = fnpf.PrismMesh(v, t, p, nz)
    eta, h, phis = C.fields(pm)
    M, En = gm.invariants(T(eta), T(h), T(phis), opts(fnpf, linear=linear))
    assert abs(M - P.mass(pm, eta)) <= 1e-13 * np.sum(np.abs(eta))
    assert abs(En - P.energy(pm, h, eta, phis, C.G, linear=linear)) <= 1e-10 * abs(En)


@pytest.mark.parametrize("p, nz, nx, ny", [(2, 2, 3, 2), (4, 2, 6, 4)])
def test_fp32_vcycle_solve_matches_oracle(fnpf, p, nz, nx, ny):
    v, t, pm = C.mesh(p, nz, nx=nx, ny=ny)
    gm = fnpf.PrismMesh(v, t, p, nz)
    eta, h, phis = C.fields(pm)
    phi64 = torch.zeros(pm.N, dtype=torch.float64, device=DEV)
    phi32 = torch.zeros(pm.N, dtype=torch.float64, device=DEV)
    i64 = gm.laplace_solve(T(eta), T(h), T(phis), phi64, opts(fnpf, pmg=True))
    i32 = gm.laplace_solve(T(eta), T(h), T(phis), phi32, opts(fnpf, pc32=True))
    assert i32["status"] == 0 and i32["rel_res"] <= 1e-13
    assert C.rel(phi32.cpu().numpy(), P.laplace_solve(pm, eta, h, phis)) <= 1e-10
    assert i32["iters"] <= i64["iters"] + 2


def test_fp32_vcycle_rk4_steps_match_oracle(fnpf):
    p, nz = 4, 2
    v, t, pm = C.mesh(p, nz, nx=4, ny=3, seed=11)
    gm = fnpf.PrismMesh(v, t, p, nz)
    eta, h, phis = C.standing_wave(pm)
    e1, p1, hd = T(eta), T(phis), T(h)
    eo, po = eta.copy(), phis.copy()
    for _ in range(3):
        gm.rk4_step(hd, e1, p1, 0.02, opts(fnpf, pc32=True))
        eo, po = P.rk4_step(pm, h, eo, po, 0.02, C.G)
    assert C.rel(e1.cpu().numpy(), eo) <= 1e-10 and C.rel(p1.cpu().numpy(), po) <= 1e-10


def test_projected_guess_same_states_fewer_iterations(fnpf):
    p, nz = 4, 2
    v, t, pm, h, cr, gen, wave = C.flume(p, nz, nx=8, ny=2)
    out = {}
    for proj in (0, 8):
        gm = fnpf.PrismMesh(v, t, p, nz)
        gm.set_relaxation(cr, gen, wave["amp"], wave["kx"], wave["ky"], wave["omega"], wave["phase"], wave["ramp_time"])
        e, ph, hd = T(np.zeros(pm.ns)), T(np.zeros(pm.ns)), T(h)
        o = fnpf.PrismMesh.default_opts(rtol=1e-12, g=C.G, precond=fnpf.FNPF_PMG, projection=proj)
        total = 0
        for k in range(6):
            total += sum(i["iters"] for i in gm.rk4_step(hd, e, ph, 0.025, o, t=4.0 + 0.025 * k))
        out[proj] = (e.cpu().numpy(), ph.cpu().numpy(), total)
    (e0, p0, n0), (e8, p8, n8) = out[0], out[8]
    assert C.rel(e8, e0) <= 1e-9 and C.rel(p8, p0) <= 1e-9
    assert n8 < 0.9 * n0, (n8, n0)


@pytest.mark.parametrize("p, nz, nx, ny", [(2, 2, 3, 2), (4, 2, 6, 4)])
def test_defect_correction_solve_matches_oracle(fnpf, p, nz, nx, ny):
    v, t, pm = C.mesh(p, nz, nx=nx, ny=ny)
    gm = fnpf.PrismMesh(v, t, p, nz)
    eta, h, phis = C.fields(pm)
    phi = torch.zeros(pm.N, dtype=torch.float64, device=DEV)
    o = fnpf.PrismMesh.default_opts(rtol=1e-13, g=C.G, precond=fnpf.FNPF_PMG, precision=fnpf.FNPF_MIXED,
                                    inner_rtol=1e-4, mass_rtol=1e-13)
    info = gm.laplace_solve(T(eta), T(h), T(phis), phi, o)
    assert info["status"] == 0 and info["rel_res"] <= 1e-13 and 1 <= info["outer_iters"] <= 6
    assert C.rel(phi.cpu().numpy(), P.laplace_solve(pm, eta, h, phis)) <= 1e-10


def test_defect_correction_rk4_steps_match_oracle(fnpf):
    p, nz = 4, 2
    v, t, pm = C.mesh(p, nz, nx=4, ny=3, seed=11)
    gm = fnpf.PrismMesh(v, t, p, nz)
    eta, h, phis = C.standing_wave(pm)
    e1, p1, hd = T(eta), T(phis), T(h)
    eo, po = eta.copy(), phis.copy()
    o = fnpf.PrismMesh.default_opts(rtol=1e-13, g=C.G, precond=fnpf.FNPF_PMG, precision=fnpf.FNPF_MIXED,
                                    mass_rtol=1e-13)
    for _ in range(3):
        gm.rk4_step(hd, e1, p1, 0.02, o)
        eo, po = P.rk4_step(pm, h, eo, po, 0.02, C.G)
    assert C.rel(e1.cpu().numpy(), eo) <= 1e-10 and C.rel(p1.cpu().numpy(), po) <= 1e-10


@pytest.mark.parametrize("p, nz, pmg", [(2, 2, False), (3, 1, True)])
def test_solve_vjp_matches_oracle_complex_step(fnpf, p, nz, pmg):
    v, t, pm = C.mesh(p, nz, nx=2, ny=1)
    gm = fnpf.PrismMesh(v, t, p, nz)
    eta, h, phis = C.fields(pm)
    phi = P.laplace_solve(pm, eta, h, phis)
    lam = np.random.default_rng(7).standard_normal(pm.N)
    le, lp, lh = (torch.zeros(pm.ns, dtype=torch.float64, device=DEV) for _ in range(3))
    gm.laplace_solve_vjp(T(eta), T(h), T(phi), T(lam), le, lp, lh, opts(fnpf, pmg=pmg))
    ge, gp, gh = C.complex_step_vjp(pm, eta, h, phis, lam)
    for dev_out, ref in ((le, ge), (lp, gp), (lh, gh)):
        assert C.rel(dev_out.cpu().numpy(), ref) <= 1e-10


@pytest.mark.parametrize("p, nz, pmg, linear", [(2, 2, False, False), (3, 1, True, False), (2, 2, True, True)])
def test_step_adjoint_matches_oracle(fnpf, p, nz, pmg, linear):
    v, t, pm = C.mesh(p, nz, nx=2, ny=1)
    gm = fnpf.PrismMesh(v, t, p, nz)
    eta, h, phis = C.fields(pm)
    rng = np.random.default_rng(3)
    le, lp = rng.standard_normal(pm.ns), rng.standard_normal(pm.ns)
    dt = 0.02
    oe, op, oh = (torch.zeros(pm.ns, dtype=torch.float64, device=DEV) for _ in range(3))
    o = fnpf.PrismMesh.default_opts(rtol=1e-13, mass_rtol=1e-13, g=C.G,
                                    precond=fnpf.FNPF_PMG if pmg else fnpf.FNPF_JACOBI,
                                    model=fnpf.FNPF_LINEAR if linear else fnpf.FNPF_NONLINEAR)
    gm.step_adjoint(T(h), T(eta), T(phis), T(le), T(lp), oe, op, dt, lam_h=oh, opts=o)
    ge, gp, gh = C.complex_step_step_vjp(pm, h, eta, phis, le, lp, dt, linear=linear)
    for dev_out, ref in ((oe, ge), (op, gp), (oh, gh)):
        assert C.rel(dev_out.cpu().numpy(), ref) <= 1e-9


def test_step_adjoint_with_relaxation_matches_oracle(fnpf):
    p, nz = 2, 1
    v, t, pm, h, cr, gen, wave = C.flume(p, nz, nx=4, ny=1)
    gm = fnpf.PrismMesh(v, t, p, nz)
    gm.set_relaxation(cr, gen, wave["amp"], wave["kx"], wave["ky"], wave["omega"], wave["phase"], wave["ramp_time"])
    rng = np.random.default_rng(9)
    x = pm.tm.xs
    eta, phis = 0.003 * np.cos(2.0 * x), 0.001 * np.sin(1.5 * x)
    le, lp = rng.standard_normal(pm.ns), rng.standard_normal(pm.ns)
    t0, dt = 4.0, 0.025
    oe, op, oh = (torch.zeros(pm.ns, dtype=torch.float64, device=DEV) for _ in range(3))
    gm.step_adjoint(T(h), T(eta), T(phis), T(le), T(lp), oe, op, dt, lam_h=oh, opts=opts(fnpf), t=t0)
    de, dp, dh = (rng.standard_normal(pm.ns) for _ in range(3))
    ce, cp = P.relaxation_step(pm, h + 1e-30j * dh, eta + 1e-30j * de, phis + 1e-30j * dp, t0, dt, C.G, cr, gen, wave)
    lhs = le @ (ce.imag / 1e-30) + lp @ (cp.imag / 1e-30)
    rhs = oe.cpu().numpy() @ de + op.cpu().numpy() @ dp + oh.cpu().numpy() @ dh
    assert abs(lhs - rhs) <= 1e-10 * abs(lhs)


def test_checkpointed_prism_gradients_match_oracle_complex_step(fnpf):
    from paper_2506_09435_gb300 import autograd as AG
    p, nz = 2, 1
    v, t, pm = C.mesh(p, nz, nx=2, ny=1)
    eta0, h0, phis0 = C.fields(pm)
    gm = fnpf.PrismMesh(v, t, p, nz)
    o = fnpf.PrismMesh.default_opts(rtol=1e-13, mass_rtol=1e-13, g=C.G)
    dt, nsteps = 0.02, 3
    e = T(eta0).requires_grad_(True)
    ph = T(phis0).requires_grad_(True)
    hh = T(h0).requires_grad_(True)
    eN, pN = AG.prism_rk4_run(gm, e, ph, hh, 0.0, dt, nsteps, every=2, opts=o)
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
        assert C.rel(grad.cpu().numpy(), ref) <= 1e-9


def test_step_adjoint_with_relaxation_and_filter_matches_oracle(fnpf):
    p, nz = 3, 1
    v, t, pm, h, cr, gen, wave = C.flume(p, nz, nx=4, ny=1)
    gm = fnpf.PrismMesh(v, t, p, nz)
    gm.set_relaxation(cr, gen, wave["amp"], wave["kx"], wave["ky"], wave["omega"], wave["phase"], wave["ramp_time"])
    gm.set_filter(4.0, 2, 1)
    rng = np.random.default_rng(11)
    x = pm.tm.xs
    eta, phis = 0.003 * np.cos(2.0 * x), 0.001 * np.sin(1.5 * x)
    le, lp = rng.standard_normal(pm.ns), rng.standard_normal(pm.ns)
    t0, dt = 4.0, 0.025
    oe, op, oh = (torch.zeros(pm.ns, dtype=torch.float64, device=DEV) for _ in range(3))
    gm.step_adjoint(T(h), T(eta), T(phis), T(le), T(lp), oe, op, dt, lam_h=oh, opts=opts(fnpf), t=t0)
    de, dp, dh = (rng.standard_normal(pm.ns) for _ in range(3))
    ce, cp = P.relaxation_step(pm, h + 1e-30j * dh, eta + 1e-30j * de, phis + 1e-30j * dp, t0, dt, C.G, cr, gen, wave,
                               filt=(4.0, 2, 1))
    lhs = le @ (ce.imag / 1e-30) + lp @ (cp.imag / 1e-30)
    rhs = oe.cpu().numpy() @ de + op.cpu().numpy() @ dp + oh.cpu().numpy() @ dh
    assert abs(lhs - rhs) <= 1e-10 * abs(lhs)
