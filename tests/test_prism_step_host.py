"""The prism solve, w, projected free-surface conditions and RK4 step of the
library (paper_2506_09435_gb300/csrc/prism_step.h: the kernels' per-thread
bodies and the host orchestration that launches them) run item by item on the
CPU through a test harness (tests/emu), against the prism oracle
(oracle/prism.py): the operator with the stored metric and its diagonal against
the assembled matrix, the Laplace solve against the direct solve, w, both
projected conditions, three RK4 steps (nonlinear and linear), special cases
(a constant surface potential, a zero right-hand side, an iteration cap), and
every entry point under AddressSanitizer (each table and workspace buffer a
separate allocation of its exact size), which checks the kernels' index
arithmetic against their buffers before their first GPU run."""
import os
import subprocess
import sys

import numpy as np
import pytest

from oracle import prism as P
from tests import prism_cases as C
from tests.emu import prism_emu as E


@pytest.fixture(scope="module")
def harness(tmp_path_factory):
    return E.Harness(E.build(str(tmp_path_factory.mktemp("prism_emu"))))


def opts(rtol=1e-13, max_iter=20000, mass_rtol=1e-14, linear=False, pmg=False, pc32=False):
    return E.opts(rtol, max_iter, mass_rtol, C.G, linear, pmg or pc32, pc32=pc32)


@pytest.mark.parametrize("p", [1, 2, 3, 4])
@pytest.mark.parametrize("nz", [1, 3])
def test_stored_operator_and_diagonal_match_oracle(harness, p, nz):
    v, t, pm = C.mesh(p, nz)
    em = harness.mesh(v, t, p, nz)
    assert (em.N, em.ns) == (pm.N, pm.ns)
    eta, h, _ = C.fields(pm)
    A = pm.assemble(eta, h)
    x = np.random.default_rng(100 + 10 * p + nz).standard_normal(pm.N)
    ref = A @ x
    assert np.max(np.abs(em.apply_stored(eta, h, x) - ref)) <= 1e-12 * np.max(np.abs(ref))
    d = A.diagonal()
    assert np.max(np.abs(em.diagonal(eta, h) - d)) <= 1e-13 * np.max(np.abs(d))


@pytest.mark.parametrize("p", [1, 2, 3, 4, 5, 6, 7, 8])
@pytest.mark.parametrize("nz", [1, 3])
def test_block_operator_equals_item_operator_bitwise(harness, p, nz):
    """The shared-memory block kernel of the operator (one prism per block, five
    phases with a barrier after each) against the one-thread-per-item kernels
    it replaces: the same arithmetic in the same order, so the same bits."""
    v, t, pm = C.mesh(p, nz, nx=2, ny=2)
    em = harness.mesh(v, t, p, nz)
    eta, h, _ = C.fields(pm)
    x = np.random.default_rng(p).standard_normal(pm.N)
    assert np.array_equal(em.apply_stored(eta, h, x), em.apply_items(eta, h, x))


@pytest.mark.parametrize("p", [1, 2, 3, 4])
def test_laplace_solve_matches_oracle(harness, p):
    nz = 2
    v, t, pm = C.mesh(p, nz)
    em = harness.mesh(v, t, p, nz)
    eta, h, phis = C.fields(pm)
    phi = np.zeros(pm.N)
    st, info = em.laplace_solve(opts(), eta, h, phis, phi)
    assert st == 0 and info.status == 0 and info.iters > 0 and info.rel_res <= 1e-13
    ref = P.laplace_solve(pm, eta, h, phis)
    assert C.rel(phi, ref) <= 1e-10
    assert np.array_equal(phi[pm.N - pm.ns:], phis)
    # warm start from the solution: converged at once, the same potential
    st, info = em.laplace_solve(opts(rtol=1e-10), eta, h, phis, phi)
    assert st == 0 and info.iters == 0 and C.rel(phi, ref) <= 1e-10


def test_solve_special_cases(harness):
    p, nz = 3, 2
    v, t, pm = C.mesh(p, nz)
    em = harness.mesh(v, t, p, nz)
    eta, h, _ = C.fields(pm)
    # a constant surface potential: the constant is harmonic with zero normal derivative
    phi = np.random.default_rng(1).standard_normal(pm.N)
    st, info = em.laplace_solve(opts(), eta, h, np.full(pm.ns, 0.3), phi)
    assert st == 0 and np.max(np.abs(phi - 0.3)) <= 1e-12
    # a zero right-hand side: phi = 0 whatever the guess, no iteration
    phi = np.random.default_rng(2).standard_normal(pm.N)
    st, info = em.laplace_solve(opts(), eta, h, np.zeros(pm.ns), phi)
    assert st == 0 and info.iters == 0 and not phi.any()
    # an iteration cap: ENOCONV, and an RK4 step leaves its state unchanged
    _, _, phis = C.fields(pm)
    st, info = em.laplace_solve(opts(max_iter=2), eta, h, phis, np.zeros(pm.N))
    assert st == 4 and info.status == 4 and info.iters == 2
    e0, p0 = eta.copy(), phis.copy()
    st, _ = em.rk4_step(opts(max_iter=2), h, e0, p0, 0.01)
    assert st == 4 and np.array_equal(e0, eta) and np.array_equal(p0, phis)


@pytest.mark.parametrize("linear", [False, True])
@pytest.mark.parametrize("p", [2, 3, 4])
def test_dtn_and_projected_conditions_match_oracle(harness, p, linear):
    nz = 2
    v, t, pm = C.mesh(p, nz)
    em = harness.mesh(v, t, p, nz)
    eta, h, phis = C.fields(pm)
    geo = np.zeros_like(eta) if linear else eta
    st, w = em.dtn(opts(linear=linear), geo, h, phis)
    assert st == 0
    assert C.rel(w, P.w_recovery(pm, geo, h, P.laplace_solve(pm, geo, h, phis))) <= 1e-10
    st, ke, kp = em.rhs(opts(linear=linear), eta, h, phis)
    assert st == 0
    ko = P.rhs(pm, h, eta, phis, C.G, linear=linear)
    assert C.rel(ke, ko[0]) <= 1e-10 and C.rel(kp, ko[1]) <= 1e-10


@pytest.mark.parametrize("linear", [False, True])
@pytest.mark.parametrize("p", [2, 4])
def test_rk4_steps_match_oracle(harness, p, linear):
    nz = 2
    v, t, pm = C.mesh(p, nz, nx=4, ny=3, seed=11)
    em = harness.mesh(v, t, p, nz)
    eta, h, phis = C.standing_wave(pm)
    e1, p1 = eta.copy(), phis.copy()
    eo, po = eta.copy(), phis.copy()
    dt = 0.02
    for _ in range(3):
        st, iters = em.rk4_step(opts(linear=linear), h, e1, p1, dt)
        assert st == 0 and max(iters) > 0
        eo, po = P.rk4_step(pm, h, eo, po, dt, C.G, linear=linear)
    assert C.rel(e1, eo) <= 1e-10 and C.rel(p1, po) <= 1e-10


@pytest.mark.parametrize("p, alpha, order, cutoff", [(3, 2.0, 2, 0), (4, 36.0, 4, 1), (5, 8.0, 2, 2), (6, 1.0, 8, 3)])
def test_modal_filter_matches_oracle(harness, p, alpha, order, cutoff):
    v, t, pm = C.mesh(p, 1)
    em = harness.mesh(v, t, p, 1)
    f = np.random.default_rng(p).standard_normal(pm.ns)
    em.set_filter(alpha, order, cutoff)
    ref = P.apply_filter(pm.tm, f, alpha, order, cutoff)
    out = em.filter_apply(f)
    assert np.max(np.abs(out - ref)) <= 1e-12 * np.max(np.abs(f))
    assert not np.array_equal(out, f)
    em.set_filter(0.0)
    with pytest.raises(AssertionError):
        em.filter_apply(f)   # no filter set: EINVAL


@pytest.mark.parametrize("p", [3, 4])
def test_filtered_rk4_steps_match_oracle(harness, p):
    nz = 2
    v, t, pm = C.mesh(p, nz, nx=4, ny=3, seed=11)
    em = harness.mesh(v, t, p, nz)
    eta, h, _ = C.standing_wave(pm)
    phis = C.fields(pm)[2]
    em.set_filter(4.0, 2, 1)
    e1, p1 = eta.copy(), phis.copy()
    eo, po = eta.copy(), phis.copy()
    for _ in range(2):
        assert em.rk4_step(opts(), h, e1, p1, 0.02)[0] == 0
        eo, po = P.rk4_step(pm, h, eo, po, 0.02, C.G)
        eo, po = P.apply_filter(pm.tm, eo, 4.0, 2, 1), P.apply_filter(pm.tm, po, 4.0, 2, 1)
    assert C.rel(e1, eo) <= 1e-10 and C.rel(p1, po) <= 1e-10


@pytest.mark.parametrize("p, nz, nx, ny", [(2, 2, 3, 2), (3, 2, 4, 3), (4, 2, 6, 4), (6, 2, 4, 3), (5, 3, 4, 3)])
def test_pmg_solve_matches_oracle_in_fewer_iterations(harness, p, nz, nx, ny):
    v, t, pm = C.mesh(p, nz, nx=nx, ny=ny)
    em = harness.mesh(v, t, p, nz)
    eta, h, phis = C.fields(pm)
    phi_j, phi_m = np.zeros(pm.N), np.zeros(pm.N)
    st, info_j = em.laplace_solve(opts(), eta, h, phis, phi_j)
    assert st == 0
    st, info_m = em.laplace_solve(opts(pmg=True), eta, h, phis, phi_m)
    assert st == 0 and info_m.rel_res <= 1e-13
    ref = P.laplace_solve(pm, eta, h, phis)
    assert C.rel(phi_m, ref) <= 1e-10
    assert info_m.iters * 3 <= info_j.iters


@pytest.mark.parametrize("p", [3, 4])
def test_vcycle_is_symmetric_positive_definite(harness, p):
    nz = 2
    v, t, pm = C.mesh(p, nz, nx=2, ny=2)
    em = harness.mesh(v, t, p, nz)
    eta, h, _ = C.fields(pm)
    NI = pm.N - pm.ns
    M = np.zeros((NI, NI))
    for j in range(NI):
        r = np.zeros(pm.N)
        r[j] = 1.0
        z = em.precond_apply(opts(pmg=True), eta, h, r)
        assert not z[NI:].any()
        M[:, j] = z[:NI]
    assert np.max(np.abs(M - M.T)) <= 1e-12 * np.max(np.abs(M))
    assert np.linalg.eigvalsh(0.5 * (M + M.T)).min() > 0


def test_pmg_rk4_steps_match_oracle(harness):
    p, nz = 4, 2
    v, t, pm = C.mesh(p, nz, nx=4, ny=3, seed=11)
    em = harness.mesh(v, t, p, nz)
    eta, h, phis = C.standing_wave(pm)
    e1, p1 = eta.copy(), phis.copy()
    eo, po = eta.copy(), phis.copy()
    for _ in range(3):
        assert em.rk4_step(opts(pmg=True), h, e1, p1, 0.02)[0] == 0
        eo, po = P.rk4_step(pm, h, eo, po, 0.02, C.G)
    assert C.rel(e1, eo) <= 1e-10 and C.rel(p1, po) <= 1e-10


@pytest.mark.parametrize("p, filt", [(2, None), (3, (4.0, 2, 1))])
def test_relaxation_zones_match_oracle(harness, p, filt):
    nz = 2
    v, t, pm, h, cr, gen, wave = C.flume(p, nz)
    em = harness.mesh(v, t, p, nz)
    em.set_relaxation(cr, gen, wave["amp"], wave["kx"], wave["ky"], wave["omega"], wave["phase"], wave["ramp_time"])
    if filt:
        em.set_filter(*filt)
    e1, p1 = np.zeros(pm.ns), np.zeros(pm.ns)
    eo, po = e1.copy(), p1.copy()
    t0, dt = 4.0, 0.025
    for k in range(3):
        assert em.rk4_step(opts(), h, e1, p1, dt, t=t0 + k * dt)[0] == 0
        eo, po = P.relaxation_step(pm, h, eo, po, t0 + k * dt, dt, C.G, cr, gen, wave, filt=filt)
    assert np.max(np.abs(eo)) > 1e-3 * wave["amp"]
    assert C.rel(e1, eo) <= 1e-10 and C.rel(p1, po) <= 1e-10


@pytest.mark.parametrize("linear", [False, True])
def test_invariants_match_oracle(harness, linear):
    p, nz = 3, 2
    v, t, pm = C.mesh(p, nz)
    em = harness.mesh(v, t, p, nz)
    eta, h, phis = C.fields(pm)
    M, En = em.invariants(opts(linear=linear), eta, h, phis)
    assert abs(M - P.mass(pm, eta)) <= 1e-13 * np.sum(np.abs(eta))
    assert abs(En - P.energy(pm, h, eta, phis, C.G, linear=linear)) <= 1e-10 * abs(En)


@pytest.mark.parametrize("p, nz, nx, ny", [(2, 2, 3, 2), (4, 2, 6, 4), (6, 2, 4, 3)])
def test_fp32_vcycle_solve_matches_oracle(harness, p, nz, nx, ny):
    """FP64 PCG with the V-cycle in FP32 (FP32 tables, metric and vectors): the
    same solution as the oracle's direct solve, in about as many iterations as
    the FP64 V-cycle."""
    v, t, pm = C.mesh(p, nz, nx=nx, ny=ny)
    em = harness.mesh(v, t, p, nz)
    eta, h, phis = C.fields(pm)
    phi64, phi32 = np.zeros(pm.N), np.zeros(pm.N)
    st, i64 = em.laplace_solve(opts(pmg=True), eta, h, phis, phi64)
    assert st == 0
    st, i32 = em.laplace_solve(opts(pc32=True), eta, h, phis, phi32)
    assert st == 0 and i32.rel_res <= 1e-13
    assert C.rel(phi32, P.laplace_solve(pm, eta, h, phis)) <= 1e-10
    assert i32.iters <= i64.iters + 2


def test_fp32_vcycle_rk4_steps_match_oracle(harness):
    p, nz = 4, 2
    v, t, pm = C.mesh(p, nz, nx=4, ny=3, seed=11)
    em = harness.mesh(v, t, p, nz)
    eta, h, phis = C.standing_wave(pm)
    e1, p1 = eta.copy(), phis.copy()
    eo, po = eta.copy(), phis.copy()
    for _ in range(3):
        assert em.rk4_step(opts(pc32=True), h, e1, p1, 0.02)[0] == 0
        eo, po = P.rk4_step(pm, h, eo, po, 0.02, C.G)
    assert C.rel(e1, eo) <= 1e-10 and C.rel(p1, po) <= 1e-10


@pytest.mark.parametrize("pmg", [False, True])
def test_projected_guess_same_states_fewer_iterations(harness, pmg):
    """The projected initial guess (the last 8 solutions and the caller's guess)
    changes where CG starts, not where it stops: six steps of the flume equal
    the unprojected run to the tolerance, in fewer iterations; an exact guess
    is kept (no iteration)."""
    p, nz = 4, 2
    v, t, pm, h, cr, gen, wave = C.flume(p, nz, nx=8, ny=2)
    out = {}
    for proj in (0, 8):
        em = harness.mesh(v, t, p, nz)
        em.set_relaxation(cr, gen, wave["amp"], wave["kx"], wave["ky"], wave["omega"], wave["phase"], wave["ramp_time"])
        e, ph = np.zeros(pm.ns), np.zeros(pm.ns)
        total = 0
        for k in range(6):
            st, it = em.rk4_step(E.opts(rtol=1e-12, g=C.G, pmg=pmg, projection=proj), h, e, ph, 0.025, t=4.0 + 0.025 * k)
            assert st == 0
            total += sum(it)
        out[proj] = (e, ph, total, em)
    (e0, p0, n0, _), (e8, p8, n8, em) = out[0], out[8]
    assert C.rel(e8, e0) <= 1e-9 and C.rel(p8, p0) <= 1e-9
    assert n8 < 0.9 * n0, (n8, n0)
    eta, hh, phis = C.fields(pm)
    ref = P.laplace_solve(pm, eta, hh, phis)
    st, info = em.laplace_solve(E.opts(rtol=1e-10, g=C.G, pmg=pmg, projection=8), eta, hh, phis, ref.copy())
    assert st == 0 and info.iters == 0


@pytest.mark.parametrize("p, nz, nx, ny", [(2, 2, 3, 2), (4, 2, 6, 4), (6, 2, 4, 3)])
def test_defect_correction_solve_matches_oracle(harness, p, nz, nx, ny):
    """FP64 defect correction around an FP32 PCG with the FP32 V-cycle: the
    oracle's solution to the FP64 tolerance, in a few outer steps."""
    v, t, pm = C.mesh(p, nz, nx=nx, ny=ny)
    em = harness.mesh(v, t, p, nz)
    eta, h, phis = C.fields(pm)
    phi = np.zeros(pm.N)
    st, info = em.laplace_solve(E.opts(rtol=1e-13, g=C.G, pmg=True, mixed=True, inner_rtol=1e-4), eta, h, phis, phi)
    assert st == 0 and info.rel_res <= 1e-13 and 1 <= info.outer_iters <= 6 and info.iters > 0
    assert C.rel(phi, P.laplace_solve(pm, eta, h, phis)) <= 1e-10


def test_defect_correction_rk4_steps_match_oracle(harness):
    p, nz = 4, 2
    v, t, pm = C.mesh(p, nz, nx=4, ny=3, seed=11)
    em = harness.mesh(v, t, p, nz)
    eta, h, phis = C.standing_wave(pm)
    e1, p1 = eta.copy(), phis.copy()
    eo, po = eta.copy(), phis.copy()
    for _ in range(3):
        assert em.rk4_step(E.opts(rtol=1e-13, g=C.G, pmg=True, mixed=True), h, e1, p1, 0.02)[0] == 0
        eo, po = P.rk4_step(pm, h, eo, po, 0.02, C.G)
    assert C.rel(e1, eo) <= 1e-10 and C.rel(p1, po) <= 1e-10


@pytest.mark.parametrize("p, nz, pmg", [(2, 2, False), (3, 1, True), (2, 3, True)])
def test_solve_vjp_matches_oracle_complex_step(harness, p, nz, pmg):
    """The vector-Jacobian product of the prism solve (adjoint solve, surface
    rows, the metric's derivative through the vertical row of J) against the
    oracle's complex-step derivatives in every eta, phis and h entry."""
    v, t, pm = C.mesh(p, nz, nx=2, ny=1)
    em = harness.mesh(v, t, p, nz)
    eta, h, phis = C.fields(pm)
    phi = P.laplace_solve(pm, eta, h, phis)
    lam = np.random.default_rng(7).standard_normal(pm.N)
    le, lp, lh = em.laplace_solve_vjp(opts(pmg=pmg), eta, h, phi, lam)
    ge, gp, gh = C.complex_step_vjp(pm, eta, h, phis, lam)
    assert C.rel(le, ge) <= 1e-10 and C.rel(lp, gp) <= 1e-10 and C.rel(lh, gh) <= 1e-10


@pytest.mark.parametrize("p, nz, pmg, linear", [(2, 2, False, False), (3, 1, True, False), (2, 2, True, True)])
def test_step_adjoint_matches_oracle(harness, p, nz, pmg, linear):
    """The adjoint of one RK4 step (forward recompute, the projected
    conditions' and w's products, the solve's VJP, the reverse RK4 sweep)
    against the oracle's complex-step tangent: the dot-product identity
    <lam, J d> = <J^T lam, d> for a random direction in (eta, phis, h), and
    J^T lam entry by entry."""
    v, t, pm = C.mesh(p, nz, nx=2, ny=1)
    em = harness.mesh(v, t, p, nz)
    eta, h, phis = C.fields(pm)
    rng = np.random.default_rng(3)
    le, lp = rng.standard_normal(pm.ns), rng.standard_normal(pm.ns)
    dt = 0.02
    st, oe, op, oh = em.step_adjoint(E.opts(rtol=1e-13, mass_rtol=1e-14, g=C.G, pmg=pmg, linear=linear), h, eta, phis,
                                     le, lp, dt)
    assert st == 0
    de, dp, dh = (rng.standard_normal(pm.ns) for _ in range(3))
    ce, cp = P.rk4_step(pm, h + 1e-30j * dh, eta + 1e-30j * de, phis + 1e-30j * dp, dt, C.G, linear=linear)
    lhs = le @ (ce.imag / 1e-30) + lp @ (cp.imag / 1e-30)
    assert abs(lhs - (oe @ de + op @ dp + oh @ dh)) <= 1e-10 * abs(lhs)
    ge, gp, gh = C.complex_step_step_vjp(pm, h, eta, phis, le, lp, dt, linear=linear)
    assert C.rel(oe, ge) <= 1e-9 and C.rel(op, gp) <= 1e-9 and C.rel(oh, gh) <= 1e-9


def test_step_adjoint_with_relaxation_matches_oracle(harness):
    """With generation and absorption zones: the dot-product identity against
    the oracle's complex-step tangent of its relaxation step (the depth's
    direction included: the target potential depends on h); with a modal
    filter the adjoint is EUNSUPPORTED."""
    p, nz = 2, 1
    v, t, pm, h, cr, gen, wave = C.flume(p, nz, nx=4, ny=1)
    em = harness.mesh(v, t, p, nz)
    em.set_relaxation(cr, gen, wave["amp"], wave["kx"], wave["ky"], wave["omega"], wave["phase"], wave["ramp_time"])
    rng = np.random.default_rng(9)
    x = pm.tm.xs
    eta, phis = 0.003 * np.cos(2.0 * x), 0.001 * np.sin(1.5 * x)
    le, lp = rng.standard_normal(pm.ns), rng.standard_normal(pm.ns)
    t0, dt = 4.0, 0.025
    st, oe, op, oh = em.step_adjoint(opts(), h, eta, phis, le, lp, dt, t=t0)
    assert st == 0
    de, dp, dh = (rng.standard_normal(pm.ns) for _ in range(3))
    ce, cp = P.relaxation_step(pm, h + 1e-30j * dh, eta + 1e-30j * de, phis + 1e-30j * dp, t0, dt, C.G, cr, gen, wave)
    lhs = le @ (ce.imag / 1e-30) + lp @ (cp.imag / 1e-30)
    assert abs(lhs - (oe @ de + op @ dp + oh @ dh)) <= 1e-10 * abs(lhs)



def test_step_adjoint_with_relaxation_and_filter_matches_oracle(harness):
    """Zones and the modal filter together (p = 3: triangles with interior
    nodes): the dot-product identity against the oracle's filtered relaxation
    step."""
    p, nz = 3, 1
    v, t, pm, h, cr, gen, wave = C.flume(p, nz, nx=4, ny=1)
    em = harness.mesh(v, t, p, nz)
    em.set_relaxation(cr, gen, wave["amp"], wave["kx"], wave["ky"], wave["omega"], wave["phase"], wave["ramp_time"])
    em.set_filter(4.0, 2, 1)
    rng = np.random.default_rng(11)
    x = pm.tm.xs
    eta, phis = 0.003 * np.cos(2.0 * x), 0.001 * np.sin(1.5 * x)
    le, lp = rng.standard_normal(pm.ns), rng.standard_normal(pm.ns)
    t0, dt = 4.0, 0.025
    st, oe, op, oh = em.step_adjoint(opts(), h, eta, phis, le, lp, dt, t=t0)
    assert st == 0
    de, dp, dh = (rng.standard_normal(pm.ns) for _ in range(3))
    ce, cp = P.relaxation_step(pm, h + 1e-30j * dh, eta + 1e-30j * de, phis + 1e-30j * dp, t0, dt, C.G, cr, gen, wave,
                               filt=(4.0, 2, 1))
    lhs = le @ (ce.imag / 1e-30) + lp @ (cp.imag / 1e-30)
    assert abs(lhs - (oe @ de + op @ dp + oh @ dh)) <= 1e-10 * abs(lhs)


ASAN_DRIVER = r"""
import sys
import numpy as np
sys.path.insert(0, sys.argv[2])
from tests import prism_cases as C
from tests.emu import prism_emu as E
hs = E.Harness(sys.argv[1])
for p, nz, nx, ny in [(1, 1, 2, 2), (3, 2, 3, 2), (5, 3, 2, 3)]:
    v, t, pm = C.mesh(p, nz, nx=nx, ny=ny)
    em = hs.mesh(v, t, p, nz)
    eta, h, phis = C.fields(pm)
    em.diagonal(eta, h)
    em.apply_stored(eta, h, np.ones(pm.N))
    em.precond_apply(E.opts(g=C.G, pmg=True), eta, h, np.ones(pm.N))
    em.precond_apply(E.opts(g=C.G, pmg=True, pc32=True), eta, h, np.ones(pm.N))
    assert em.laplace_solve(E.opts(g=C.G, pmg=True, pc32=True), eta, h, phis, np.zeros(pm.N))[0] == 0
    o = E.opts(g=C.G, pmg=(p > 1))
    assert em.laplace_solve(o, eta, h, phis, np.zeros(pm.N))[0] == 0
    assert em.dtn(o, eta, h, phis)[0] == 0
    assert em.rhs(o, eta, h, phis)[0] == 0
    assert em.rk4_step(o, h, eta, phis, 0.01)[0] == 0
    em.invariants(o, eta, h, phis)
    o.model = 1
    assert em.rk4_step(o, h, eta, phis, 0.01)[0] == 0
    if p >= 3:
        em.set_filter(2.0, 2, 1)
        em.filter_apply(eta)
        assert em.rk4_step(o, h, eta, phis, 0.01)[0] == 0
# the edges of the valid range: one level (p = 1), four levels (p = 8), one layer; every option at once
for p, nz in [(1, 1), (8, 1), (7, 2)]:
    v, t, pm = C.mesh(p, nz, nx=2, ny=1)
    em = hs.mesh(v, t, p, nz)
    eta, h, phis = C.fields(pm)
    for o in (E.opts(g=C.G, pmg=True), E.opts(g=C.G, pmg=True, pc32=True), E.opts(g=C.G, pmg=True, linear=True),
              E.opts(g=C.G, pmg=True, mixed=True, projection=8)):
        assert em.laplace_solve(o, eta, h, phis, np.zeros(pm.N))[0] == 0
        assert em.rk4_step(o, h, eta.copy(), phis.copy(), 0.01)[0] == 0
    em.invariants(E.opts(g=C.G, pmg=True, pc32=True), eta, h, phis)
    em.laplace_solve_vjp(E.opts(g=C.G, pmg=True), eta, h, np.ones(pm.N), np.ones(pm.N))
    assert em.step_adjoint(E.opts(g=C.G, pmg=True), h, eta, phis, np.ones(pm.ns), np.ones(pm.ns), 0.01)[0] == 0
    for k in range(3):
        assert em.rk4_step(E.opts(g=C.G, pmg=True, projection=8), h, eta.copy(), phis.copy(), 0.01)[0] == 0
v, t, pm, h, cr, gen, wave = C.flume(4, 2, nx=4, ny=1)
em = hs.mesh(v, t, 4, 2)
em.set_filter(4.0, 2, 1)
em.set_relaxation(cr, gen, wave["amp"], wave["kx"], wave["ky"], wave["omega"], wave["phase"], wave["ramp_time"])
assert em.rk4_step(E.opts(g=C.G, pmg=True, pc32=True), h, np.zeros(pm.ns), np.zeros(pm.ns), 0.02, t=4.0)[0] == 0
v, t, pm, h, cr, gen, wave = C.flume(3, 2, nx=4, ny=1)
em = hs.mesh(v, t, 3, 2)
em.set_relaxation(cr, gen, wave["amp"], wave["kx"], wave["ky"], wave["omega"], wave["phase"], wave["ramp_time"])
assert em.rk4_step(E.opts(g=C.G), h, np.zeros(pm.ns), np.zeros(pm.ns), 0.02, t=4.0)[0] == 0
print("asan run ok")
"""


def test_every_entry_point_in_bounds_under_asan(tmp_path):
    rt = E.asan_runtime()
    if rt is None:
        pytest.skip("no AddressSanitizer runtime")
    lib = E.build(str(tmp_path), asan=True)
    env = dict(os.environ, LD_PRELOAD=rt, ASAN_OPTIONS="detect_leaks=0:abort_on_error=0")
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    r = subprocess.run([sys.executable, "-c", ASAN_DRIVER, lib, root], capture_output=True, text=True, env=env,
                       timeout=600)
    assert r.returncode == 0 and "AddressSanitizer" not in r.stderr, r.stderr[-4000:]
    assert "asan run ok" in r.stdout
