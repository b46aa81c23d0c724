"""Differentiable RK4 time loop (torch.autograd.Function) with checkpointing.

Forward: `nsteps` calls of fnpf_rk4_step on one work buffer, storing (eta,
phi_eta) every `every` steps.  Backward: for each segment, newest first, the
segment is recomputed from its checkpoint with the mesh's tape recording the
stage states and potentials of each step (fnpf_tape_begin), and
fnpf_step_adjoint_taped runs over its steps in reverse, accumulating dJ/dh, so
no forward solve is repeated inside the adjoint steps.  Every computation runs
in libfnpf's kernels; this module only orders the calls.
"""
import torch


class RK4Run(torch.autograd.Function):
    @staticmethod
    def forward(ctx, eta0, phis0, h, mesh, t0, dt, nsteps, every):
        work_e = eta0.detach().clone().contiguous()
        work_p = phis0.detach().clone().contiguous()
        ckpts = []
        for n in range(nsteps):
            if n % every == 0:
                ckpts.append((n, work_e.clone(), work_p.clone()))
            mesh.rk4_step(work_e, work_p, t0 + n * dt, dt)
        ctx.mesh, ctx.t0, ctx.dt, ctx.nsteps, ctx.every = mesh, t0, dt, nsteps, every
        ctx.ckpts, ctx.work = ckpts, (work_e, work_p)
        ctx.h_shape = h.shape
        return work_e.clone(), work_p.clone()

    @staticmethod
    def backward(ctx, g_eta, g_phis):
        mesh, t0, dt, nsteps, every = ctx.mesh, ctx.t0, ctx.dt, ctx.nsteps, ctx.every
        work_e, work_p = ctx.work
        lam_e = (g_eta if g_eta is not None else torch.zeros_like(work_e)).detach().clone().contiguous()
        lam_p = (g_phis if g_phis is not None else torch.zeros_like(work_p)).detach().clone().contiguous()
        lam_h = torch.zeros(ctx.h_shape, dtype=lam_e.dtype, device=lam_e.device)
        for n0, e0, p0 in reversed(ctx.ckpts):
            n1 = min(n0 + every, nsteps)
            work_e.copy_(e0)
            work_p.copy_(p0)
            mesh.tape_begin(n1 - n0)
            try:
                for n in range(n0, n1):
                    mesh.rk4_step(work_e, work_p, t0 + n * dt, dt)
            finally:
                mesh.tape_end()
            for n in reversed(range(n0, n1)):
                mesh.step_adjoint_taped(n - n0, lam_e, lam_p, lam_e, lam_p, lam_h, dt)
        return lam_e, lam_p, lam_h, None, None, None, None, None


def rk4_run(mesh, eta0, phis0, h, t0, dt, nsteps, every=16):
    """(eta_N, phi_N) after nsteps RK4 steps; differentiable in eta0, phis0 and h
    (the gradient for h is dJ/dh at the surface nodes).

    The forward runs on the depth the mesh was created with, so `h` must be
    that depth (the same values, [Ns] doubles): it is the handle through which
    autograd reports dJ/dh, and a different h would label the gradient of one
    depth with another.  A mismatch raises ValueError."""
    _check_depth(mesh, h)
    return RK4Run.apply(eta0, phis0, h, mesh, t0, dt, nsteps, every)


def _check_depth(mesh, h):
    mesh_h = mesh.depth()
    if tuple(h.shape) != (mesh.ns,):
        raise ValueError("h must have the mesh's %d surface nodes, got shape %s" % (mesh.ns, tuple(h.shape)))
    hd = h.detach().to(device="cpu", dtype=torch.float64)
    if not torch.equal(hd, mesh_h):
        raise ValueError("h differs from the depth the mesh was created with (max |difference| %.3e); "
                         "create a mesh with this depth instead" % float((hd - mesh_h).abs().max()))


class RK4Trajectory(torch.autograd.Function):
    """The states after steps keep_from, ..., nsteps of an RK4 run, stacked
    ([K, Ns] each), differentiable in eta0, phis0 and h: the reverse sweep adds
    the cotangent of every kept state as it passes that step (the adjoint of a
    time-integrated objective).  Checkpoints every `every` steps, segments
    recomputed with the tape, as in RK4Run."""

    @staticmethod
    def forward(ctx, eta0, phis0, h, mesh, t0, dt, nsteps, keep_from, every):
        work_e = eta0.detach().clone().contiguous()
        work_p = phis0.detach().clone().contiguous()
        ckpts, kept_e, kept_p = [], [], []
        for n in range(nsteps + 1):
            if n >= keep_from:
                kept_e.append(work_e.clone())
                kept_p.append(work_p.clone())
            if n == nsteps:
                break
            if n % every == 0:
                ckpts.append((n, work_e.clone(), work_p.clone()))
            mesh.rk4_step(work_e, work_p, t0 + n * dt, dt)
        ctx.mesh, ctx.t0, ctx.dt, ctx.nsteps, ctx.keep_from, ctx.every = mesh, t0, dt, nsteps, keep_from, every
        ctx.ckpts, ctx.work = ckpts, (work_e, work_p)
        ctx.h_shape = h.shape
        return torch.stack(kept_e), torch.stack(kept_p)

    @staticmethod
    def backward(ctx, g_eta, g_phis):
        mesh, t0, dt, nsteps, k0, every = ctx.mesh, ctx.t0, ctx.dt, ctx.nsteps, ctx.keep_from, ctx.every
        work_e, work_p = ctx.work
        K = nsteps - k0 + 1
        g_eta = g_eta if g_eta is not None else torch.zeros((K,) + work_e.shape, dtype=work_e.dtype,
                                                            device=work_e.device)
        g_phis = g_phis if g_phis is not None else torch.zeros_like(g_eta)
        lam_e = g_eta[K - 1].detach().clone().contiguous()
        lam_p = g_phis[K - 1].detach().clone().contiguous()
        lam_h = torch.zeros(ctx.h_shape, dtype=lam_e.dtype, device=lam_e.device)
        for n0, e0, p0 in reversed(ctx.ckpts):
            n1 = min(n0 + every, nsteps)
            work_e.copy_(e0)
            work_p.copy_(p0)
            mesh.tape_begin(n1 - n0)
            try:
                for n in range(n0, n1):
                    mesh.rk4_step(work_e, work_p, t0 + n * dt, dt)
            finally:
                mesh.tape_end()
            for n in reversed(range(n0, n1)):
                mesh.step_adjoint_taped(n - n0, lam_e, lam_p, lam_e, lam_p, lam_h, dt)
                if n >= k0:
                    lam_e += g_eta[n - k0]
                    lam_p += g_phis[n - k0]
        return lam_e, lam_p, lam_h, None, None, None, None, None, None


def rk4_trajectory(mesh, eta0, phis0, h, t0, dt, nsteps, keep_from=0, every=16):
    """(etas, phiss) [K, Ns]: the states after steps keep_from .. nsteps of an
    RK4 run (K = nsteps - keep_from + 1), differentiable in eta0, phis0 and h;
    h must be the depth the mesh was created with (as for rk4_run)."""
    if not 0 <= keep_from <= nsteps:
        raise ValueError("need 0 <= keep_from <= nsteps")
    _check_depth(mesh, h)
    return RK4Trajectory.apply(eta0, phis0, h, mesh, t0, dt, nsteps, keep_from, every)

class PrismRK4Run(torch.autograd.Function):
    """The RK4 loop on a prism mesh (fnpf_prism_rk4_step forward,
    fnpf_prism_step_adjoint backward) with checkpoints every `every` steps:
    the backward recomputes each segment's step-start states from its
    checkpoint, newest segment first, and runs the step adjoints over them in
    reverse, accumulating dJ/dh (the depth enters every call, so it is
    differentiated directly)."""

    @staticmethod
    def forward(ctx, eta0, phis0, h, mesh, t0, dt, nsteps, every, opts):
        work_e = eta0.detach().clone().contiguous()
        work_p = phis0.detach().clone().contiguous()
        hd = h.detach().contiguous()
        ckpts = []
        for n in range(nsteps):
            if n % every == 0:
                ckpts.append((n, work_e.clone(), work_p.clone()))
            mesh.rk4_step(hd, work_e, work_p, dt, opts, t=t0 + n * dt)
        ctx.mesh, ctx.t0, ctx.dt, ctx.nsteps, ctx.every, ctx.opts = mesh, t0, dt, nsteps, every, opts
        ctx.ckpts, ctx.hd = ckpts, hd
        return work_e.clone(), work_p.clone()

    @staticmethod
    def backward(ctx, g_eta, g_phis):
        mesh, t0, dt, nsteps, every, opts, hd = ctx.mesh, ctx.t0, ctx.dt, ctx.nsteps, ctx.every, ctx.opts, ctx.hd
        ref = ctx.ckpts[0][1]
        lam_e = (g_eta if g_eta is not None else torch.zeros_like(ref)).detach().clone().contiguous()
        lam_p = (g_phis if g_phis is not None else torch.zeros_like(ref)).detach().clone().contiguous()
        out_e, out_p = torch.empty_like(lam_e), torch.empty_like(lam_p)
        lam_h = torch.zeros_like(hd)
        step_h = torch.empty_like(hd)
        for n0, e0, p0 in reversed(ctx.ckpts):
            n1 = min(n0 + every, nsteps)
            states = [(e0.clone(), p0.clone())]
            for n in range(n0, n1 - 1):
                e, p = states[-1][0].clone(), states[-1][1].clone()
                mesh.rk4_step(hd, e, p, dt, opts, t=t0 + n * dt)
                states.append((e, p))
            for n in reversed(range(n0, n1)):
                e, p = states[n - n0]
                mesh.step_adjoint(hd, e, p, lam_e, lam_p, out_e, out_p, dt, lam_h=step_h, opts=opts, t=t0 + n * dt)
                lam_e, out_e = out_e, lam_e
                lam_p, out_p = out_p, lam_p
                lam_h += step_h
        return lam_e, lam_p, lam_h, None, None, None, None, None, None


def prism_rk4_run(mesh, eta0, phis0, h, t0, dt, nsteps, every=16, opts=None):
    """(eta_N, phi_N) after nsteps RK4 steps on a prism mesh (PrismMesh);
    differentiable in eta0, phis0 and the depth h [Ns]."""
    return PrismRK4Run.apply(eta0, phis0, h, mesh, t0, dt, nsteps, every, opts)
