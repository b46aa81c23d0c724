#!/usr/bin/env python
"""Throughput benchmark of the FNPF-SEM hot path on GB300.

One step = one classical RK4 step of the fully nonlinear free-surface state:
four Laplace solves on the eta-following mesh, four vertical-velocity
recoveries and Zakharov right-hand sides, the RK4 combination.

Workload: the 3D nonlinear periodic box, flat bottom, kh = 2, 32 x 32 x 2
hexahedra of GLL order 6 (479,232 volume DOF), Airy wave H/L = 0.05 plus a
seeded Gaussian spectrum of perturbations (seed 2), dt = T/100, Laplace solves
to rtol 1e-10.  Metric: DOF x RK4 steps per second (DOF = global volume
nodes), whole job over all ranks.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gb300|reference]

--impl reference times the FP64 CPU oracle (the slow, obviously-correct
restatement used by the tests) on the host cores, on a bounded sample of the
same workload, and prints the same JSON line with "impl": "reference".
"""
import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "DOF·RK4-steps/s at 1e-8 rel error, FP64 vs mixed-precision; adjoint cost ratio"
UNIT = "DOF·steps/s"
WORKLOAD = "periodic-box-3d kh=2, 32x32x2 hex, GLL p=6, Airy H/L=0.05 + seeded spectrum, dt=T/100, rtol 1e-10"
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.070e9 / 1e12   # 152 SMs x 2 DFMA/clk x 2 flop x 2070 MHz
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.070e9 / 1e12  # 152 SMs x 128 FFMA/clk x 2 flop x 2070 MHz
# ncu dram__bytes_read.sum + dram__bytes_write.sum of one launch of the FP64 stored-metric operator on the
# benchmark tank (kernel alone, cold cache): axg_kernel<double,7,3,7> (shape 3), axl_kernel<double,7,7,1> (shape 4)
AXG_C2_DRAM_BYTES = 34.060544e6 + 768.0
AXL_C2_DRAM_BYTES = 37.302272e6 + 768.0


def measured_hbm_gbs():
    """Measured copy bandwidth of this GPU model (MEASURED_PEAKS.json beside
    this file), else the figure measured earlier on the same model."""
    try:
        with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"])
    except (OSError, KeyError, ValueError):
        return 6785.2


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--rtol", type=float, default=1e-10)
    ap.add_argument("--precond", default="pmg", choices=["pmg", "jacobi"])
    ap.add_argument("--cheb-degree", type=int, default=3, help="Chebyshev degree of the FP64 path's smoothers")
    ap.add_argument("--mixed-cheb-degree", type=int, default=3, help="... of the mixed path's FP32 smoothers")
    ap.add_argument("--coarse-degree", type=int, default=6)
    ap.add_argument("--shape", type=int, default=-1, choices=list(range(-1, 12)),
                    help="elements-per-CTA shape of the operator kernels (-1: autotuned)")
    ap.add_argument("--shapes", default="", help="FP64,FP32 elements-per-CTA shapes of the headline mesh "
                    "(e.g. 4,3; default: autotuned, or --shape)")
    ap.add_argument("--model", default="fnpf", choices=["fnpf", "lpf"],
                    help="fnpf: fully nonlinear (the configuration's method); lpf: linear potential flow")
    ap.add_argument("--mg-schedule", default="halve", choices=["halve", "two", "step2"],
                    help="multigrid orders: p, p/2, ..., 1 (halve); p, 1 (two); p, p-2, ..., 1 (step2)")
    ap.add_argument("--cheb-kind", type=int, default=1, choices=[1, 4],
                    help="Chebyshev smoother: 1 = first kind on [lmax/20, lmax], 4 = fourth kind on [0, lmax]")
    ap.add_argument("--cheb-range", type=float, default=160.0,
                    help="first-kind Chebyshev smoothers target [lmax / range, lmax]")
    ap.add_argument("--coarse-solver", default="cluster", choices=["cluster", "launches"],
                    help="coarsest multigrid level on one thread-block cluster, or one launch per step")
    ap.add_argument("--inner-rtol", type=float, default=1e-4,
                    help="relative tolerance of the FP32 inner solves of the defect-correction form (with the "
                         "projected initial guess, 1e-4 needs one outer step, as 1e-5 did, with fewer inner "
                         "iterations)")
    ap.add_argument("--projection", type=int, default=8,
                    help="initial guess of each solve projected onto the last N solutions (0: previous solution)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-mixed", action="store_true")
    ap.add_argument("--no-adjoint", action="store_true")
    ap.add_argument("--no-prism", action="store_true", help="skip the prism-mesh leg of the step benchmark")
    ap.add_argument("--no-bar", action="store_true", help="skip the shortened bar-flume leg of the step benchmark")
    ap.add_argument("--precision", default="fp64", choices=["fp64", "mixed", "pc32"],
                    help="precision of the headline path (the configuration's plain method is fp64)")
    ap.add_argument("--nx", type=int, default=32)
    ap.add_argument("--mode", default="step",
                    choices=["step", "apply", "ensemble", "convergence", "bar", "cylinder", "peaks", "prism"],
                    help="step: RK4 steps (the benchmark); apply: operator applications only; "
                         "ensemble: 64 seeded tanks in one launch per step vs one tank at a time; "
                         "convergence: error of a stream-function wave after one period vs p and h; "
                         "bar: the submerged-bar flume in FP64 and both mixed-precision forms; "
                         "cylinder: adjoint cost on the O-grid around a cylinder; "
                         "peaks: measured FP64 / FP32 FMA throughput; "
                         "prism: the prism-mesh leg (triangulated flume) alone")
    ap.add_argument("--tanks", type=int, default=64)
    ap.add_argument("--bar-steps", type=int, default=150, help="RK4 steps of the bar-flume accuracy run")
    ap.add_argument("--p", type=int, default=6)
    ap.add_argument("--nz", type=int, default=2)
    return ap.parse_args()


def workload(nx=32):
    from paper_2506_09435_gb300 import workloads as W
    return W.periodic_box_3d(nx=nx, ny=nx, nz=2, p=6, kh=2.0)


# ----------------------------------------------------------------------------- oracle legs

ORACLE_SAMPLE = """
import json, sys, time
sys.path.insert(0, {root!r})
import numpy as np
from oracle import mesh, surface
from paper_2506_09435_gb300 import workloads as W
nxy, steps, warm, out = {nxy}, {steps}, {warm}, {out!r}
d = W.periodic_box_3d(nx=nxy, ny=nxy, nz=2, p=6, kh=2.0)
m = mesh.Mesh(3, nxy, nxy, 2, 6, True, True, d['Lx'], d['Ly'])
x, y = m.surface_coords()
h = np.full(m.ns, d['h0'])
eta, phis = W.airy_plus_spectrum_state(d, x, y, seed=2)
dt = W.period(d['k'], d['h0'], d['g']) / 100
for _ in range(warm):
    eta, phis = surface.rk4_step(m, h, eta, phis, dt, d['g'], method='pcg')
times = []
for _ in range(steps):
    t0 = time.perf_counter()
    eta, phis = surface.rk4_step(m, h, eta, phis, dt, d['g'], method='pcg')
    times.append(time.perf_counter() - t0)
if out:
    np.savez(out, eta=eta, phis=phis)
print(json.dumps(dict(N=m.N, times=times)))
"""

ONE_THREAD = dict(OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")

PRISM_ORACLE_SAMPLE = """
import json, sys, time
sys.path.insert(0, {root!r})
import numpy as np
from oracle import prism as P
from paper_2506_09435_gb300 import workloads as W
v, t, d = W.prism_flume(nx={nx}, ny={ny}, p={p}, nz={nz})
pm = P.PrismMesh(P.TriMesh(v, t, d['p']), d['nz'])
cr, gen = W.flume_zones(d, pm.tm.xs)
wave = W.flume_wave(d)
h = np.full(pm.ns, d['h0'])
eta, phis = np.zeros(pm.ns), np.zeros(pm.ns)
t0, dt = {t0}, d['T'] / 40
times = []
for k in range({steps}):
    s = time.perf_counter()
    eta, phis = P.relaxation_step(pm, h, eta, phis, t0 + k * dt, dt, d['g'], cr, gen, wave)
    times.append(time.perf_counter() - s)
np.savez({out!r}, eta=eta, phis=phis)
print(json.dumps(dict(N=pm.N, times=times)))
"""


def run_oracle_sample(nxy, steps, warm, out=""):
    """The oracle on the sample tank in a child process with one thread;
    with `out`, the state after warm + steps RK4 steps is saved there (npz)."""
    env = dict(os.environ, **ONE_THREAD)
    code = ORACLE_SAMPLE.format(root=ROOT, nxy=nxy, steps=steps, warm=warm, out=out)
    res = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, check=True)
    return json.loads(res.stdout.strip().splitlines()[-1])


def run_oracle_replicas(nxy, steps, procs):
    """`procs` copies of the oracle sample at once, one thread each (the host's
    cores busy with independent tanks, as replicas of the workload); returns
    the aggregate DOF x steps / s over the slowest copy's timed steps."""
    env = dict(os.environ, **ONE_THREAD)
    code = ORACLE_SAMPLE.format(root=ROOT, nxy=nxy, steps=steps, warm=0, out="")
    ps = [subprocess.Popen([sys.executable, "-c", code], env=env, stdout=subprocess.PIPE,
                           stderr=subprocess.DEVNULL, text=True) for _ in range(procs)]
    res = []
    for p in ps:
        o, _ = p.communicate()
        if p.returncode != 0:
            raise RuntimeError("oracle replica failed")
        res.append(json.loads(o.strip().splitlines()[-1]))
    slowest = max(sum(r["times"]) for r in res)
    return procs * res[0]["N"] * steps / slowest, res[0]["N"]


def host_cpu():
    """nproc and the CPU model of this host (lscpu, else /proc/cpuinfo)."""
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                model = line.split(":", 1)[1].strip()
                break
    except Exception:
        pass
    if model is None:
        try:
            for line in open("/proc/cpuinfo"):
                if line.lower().startswith("model name"):
                    model = line.split(":", 1)[1].strip()
                    break
        except OSError:
            pass
    return {"nproc": os.cpu_count(), "model": model}


def oracle_sample_desc(nxy, steps):
    return ("FP64 numpy/scipy oracle, 1 thread: %d RK4 step(s) of the same tank shape reduced to %dx%dx2 "
            "elements (p=6, kh=2, same seeded state), Jacobi-CG to rtol 1e-14 on the assembled sparse matrix"
            % (steps, nxy, nxy))


class Ranks:
    """Ranks of a torchrun launch (RANK, LOCAL_RANK, WORLD_SIZE from the
    environment): one process per GPU, each timing its own tank (replicas, no
    data-path collective); the only collectives are barriers and the maximum
    over ranks of a timing."""

    def __init__(self, backend="nccl"):
        self.world = int(os.environ.get("WORLD_SIZE", "1"))
        self.rank = int(os.environ.get("RANK", "0"))
        self.local = int(os.environ.get("LOCAL_RANK", "0"))
        self.dist = None
        if self.world > 1:
            import torch.distributed as dist
            if backend == "nccl":
                # bind this rank to its own GPU before the process group
                # exists, so that NCCL's barriers and reductions use it
                import torch
                torch.cuda.set_device(self.local)
            dist.init_process_group(backend)
            self.dist = dist

    def barrier(self):
        if self.dist is not None:
            self.dist.barrier()

    def max(self, value, device):
        """The largest value over all ranks (the job's time is its slowest rank's)."""
        if self.dist is None:
            return value
        import torch
        t = torch.tensor([value], dtype=torch.float64, device=device)
        self.dist.all_reduce(t, op=self.dist.ReduceOp.MAX)
        return float(t.item())

    def close(self):
        if self.dist is not None:
            self.dist.destroy_process_group()


def main_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    nxy = 4
    res = run_oracle_sample(nxy, args.steps, args.warmup)
    total = sum(res["times"])
    value = res["N"] * args.steps / total
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "sample": "%dx%dx2 elements, N=%d" % (nxy, nxy, res["N"])},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": oracle_sample_desc(nxy, args.steps)},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


# ----------------------------------------------------------------------------- FMA peaks

def measure_fma_peaks(dev, reps=5):
    """Measured FP64 and FP32 FMA throughput (fnpf_fma_probe: 8 independent
    FMA chains per thread, 16 CTAs of 256 threads per SM), best of `reps`
    launches timed with CUDA events on the launching stream, TFLOP/s."""
    import torch

    from paper_2506_09435_gb300 import fnpf
    stream = torch.cuda.current_stream()
    out = {}
    for name, prec, dtype, iters in (("fp64", fnpf.FNPF_FP64, torch.float64, 400),
                                     ("fp32", fnpf.FNPF_MIXED, torch.float32, 8000)):
        buf = torch.zeros(1, dtype=dtype, device=dev)
        blocks = 152 * 16
        fnpf.fma_probe(prec, blocks, iters, buf)
        best = None
        for _ in range(reps):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            flops = fnpf.fma_probe(prec, blocks, iters, buf)
            b.record(stream)
            torch.cuda.synchronize()
            ms = a.elapsed_time(b)
            best = ms if best is None else min(best, ms)
        out[name] = {"tflops": flops / (best * 1e-3) / 1e12, "ms": best, "flops": flops}
    return out


# ----------------------------------------------------------------------------- clocks

CLOCK_QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
               "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
               "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")


class ClockSampler:
    def __init__(self, index):
        self.index = index
        self.proc = None
        # raw samples go to a temporary file; their summary is part of the JSON line
        self.path = os.path.join(tempfile.gettempdir(), "fnpf_bench_clocks_%d.csv" % os.getpid())

    def __enter__(self):
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + CLOCK_QUERY,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.f.close()

    def summary(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [v.strip() for v in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ----------------------------------------------------------------------------- GPU arm

def main_gb300(args):
    import numpy as np
    import torch

    from paper_2506_09435_gb300 import fnpf
    from paper_2506_09435_gb300 import workloads as W

    ranks = Ranks("nccl")
    world, rank, local = ranks.world, ranks.rank, ranks.local
    torch.cuda.set_device(local)
    barrier = ranks.barrier

    d = workload(args.nx)
    h = None
    pre = fnpf.FNPF_PMG if args.precond == "pmg" else fnpf.FNPF_JACOBI
    prec = {"fp64": fnpf.FNPF_FP64, "mixed": fnpf.FNPF_MIXED, "pc32": fnpf.FNPF_FP64_PC32}[args.precision]
    cdeg = args.mixed_cheb_degree if args.precision == "mixed" else args.cheb_degree
    opts = fnpf.default_opts(rtol=args.rtol, max_iter=50000, precond=pre, cheb_degree=cdeg,
                             coarse_iters=args.coarse_degree, coarse_solver=coarse_mode(args),
                             cheb_kind=args.cheb_kind, cheb_range=args.cheb_range,
                             model=model_id(args), mg_schedule=schedule_id(args),
                             precision=prec, projection=args.projection, inner_rtol=args.inner_rtol)
    ncx = d["p"] * d["nx"]
    h = np.full(ncx * ncx, d["h0"])
    mesh = fnpf.Mesh(3, d["nx"], d["ny"], d["nz"], d["p"], True, True, h, Lx=d["Lx"], Ly=d["Ly"], g=d["g"],
                     opts=opts)
    if args.shape >= 0:
        mesh.set_shapes(args.shape, args.shape)
    if args.shapes:
        mesh.set_shapes(*[int(v) for v in args.shapes.split(",")])
    x, y = mesh.surface_coords()
    eta0, phi0 = W.airy_plus_spectrum_state(d, x, y, seed=2)
    dt = W.period(d["k"], d["h0"], d["g"]) / 100
    dev = torch.device("cuda", local)
    eta = torch.tensor(eta0, dtype=torch.float64, device=dev)
    phis = torch.tensor(phi0, dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream()
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)   # 256 MB > L2 (129 MB)
    t = 0.0
    for _ in range(args.warmup):
        mesh.rk4_step(eta, phis, t, dt)
        t += dt
    torch.cuda.synchronize()

    # --- timed region: K RK4 steps, L2 flushed before each, device time per step
    eta_start, phi_start = eta.clone(), phis.clone()     # for the mass and energy drift over the timed steps
    mesh.profile_read(reset=True)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    infos = []
    with ClockSampler(local) as clk:
        barrier()
        torch.cuda.synchronize()
        wall0 = time.perf_counter()
        for k in range(args.steps):
            flush.zero_()
            ev[k][0].record(stream)
            infos.append(mesh.rk4_step(eta, phis, t, dt, info=True))
            ev[k][1].record(stream)
            t += dt
        torch.cuda.synchronize()
        barrier()
        wall = time.perf_counter() - wall0
    launches = mesh.profile_read(reset=True)["launches"]
    eta64_end, phi64_end = eta.clone(), phis.clone()
    # conserved quantities before and after the timed steps (fnpf_invariants, outside the timed region)
    m0, e0 = mesh.invariants(eta_start, phi_start)
    m1, e1 = mesh.invariants(eta64_end, phi64_end)
    wave_h = 0.05 * 2 * math.pi / d["k"]          # H = steepness x wavelength
    drift = {"steps": args.steps, "mass_start": m0, "mass_end": m1, "energy_start": e0, "energy_end": e1,
             "mass_drift_over_H_area": abs(m1 - m0) / (wave_h * d["Lx"] * d["Ly"]),
             "energy_drift_rel": abs(e1 - e0) / abs(e0),
             "how": "M = sum W eta, E = 1/2 phi^T A phi + 1/2 g sum W eta^2 (lumped GLL mass W), fnpf_invariants"}
    step_ms = [a.elapsed_time(b) for a, b in ev]
    total_ms = sum(step_ms)
    total_ms = ranks.max(total_ms, dev)
    value = world * mesh.N * args.steps / (total_ms * 1e-3)
    iters = [i["iters"] for inf in infos for i in inf]
    rel_res = max(i["rel_res"] for inf in infos for i in inf)
    assert all(i["status"] == 0 for inf in infos for i in inf)
    assert torch.isfinite(eta).all() and torch.isfinite(phis).all()

    # --- the other precision forms on the same workload from the same initial state, each
    #     reported with its error against the FP64 path: FNPF_MIXED (FP64 defect correction
    #     around an FP32 operator, FP32 p-MG and FP32 PCG) and FNPF_FP64_PC32 (FP64 PCG with
    #     the p-MG preconditioner in FP32)
    def precision_form(prec_id, cheb):
        mopts = fnpf.default_opts(precision=prec_id, rtol=args.rtol, inner_rtol=args.inner_rtol, max_iter=50000,
                                  precond=pre, cheb_degree=cheb, coarse_iters=args.coarse_degree,
                                  coarse_solver=coarse_mode(args), cheb_kind=args.cheb_kind,
                                  cheb_range=args.cheb_range, model=model_id(args), mg_schedule=schedule_id(args),
                                  projection=args.projection)
        mm = fnpf.Mesh(3, d["nx"], d["ny"], d["nz"], d["p"], True, True, h, Lx=d["Lx"], Ly=d["Ly"], g=d["g"],
                       opts=mopts)
        if args.shape >= 0:
            mm.set_shapes(args.shape, args.shape)
        em = torch.tensor(eta0, dtype=torch.float64, device=dev)
        pm = torch.tensor(phi0, dtype=torch.float64, device=dev)
        tm = 0.0
        for _ in range(args.warmup):
            mm.rk4_step(em, pm, tm, dt)
            tm += dt
        torch.cuda.synchronize()
        mm.profile_read(reset=True)
        mev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
               for _ in range(args.steps)]
        minfos = []
        barrier()
        torch.cuda.synchronize()
        for k in range(args.steps):
            flush.zero_()
            mev[k][0].record(stream)
            minfos.append(mm.rk4_step(em, pm, tm, dt, info=True))
            mev[k][1].record(stream)
            tm += dt
        torch.cuda.synchronize()
        barrier()
        mlaunch = mm.profile_read(reset=True)["launches"]
        m_ms = sum(a.elapsed_time(b) for a, b in mev)
        m_ms = ranks.max(m_ms, dev)
        err_e = float(torch.linalg.norm(em - eta64_end) / torch.linalg.norm(eta64_end))
        err_p = float(torch.linalg.norm(pm - phi64_end) / torch.linalg.norm(phi64_end))
        mm.profile_enable(True)
        for _ in range(2):
            flush.zero_()
            mm.rk4_step(em, pm, tm, dt)
            tm += dt
        torch.cuda.synchronize()
        mprof = mm.profile_read(reset=True)
        out = {"value": world * mesh.N * args.steps / (m_ms * 1e-3), "unit": UNIT,
               "ms_per_step": m_ms / args.steps,
               "dtype": "f32 inner / f64 outer" if prec_id == fnpf.FNPF_MIXED
               else "f64 PCG, f32 p-multigrid preconditioner",
               "cheb_degree": cheb,
               "rel_l2_vs_fp64_path": {"eta": err_e, "phis": err_p},
               "inner_iters_per_solve_mean": statistics.mean(i["iters"] for inf in minfos for i in inf),
               "outer_iters_per_solve_mean": statistics.mean(i["outer_iters"] for inf in minfos for i in inf),
               "max_rel_res": max(i["rel_res"] for inf in minfos for i in inf),
               "fp32_apply_ms": mprof["apply32_ms"] / max(1, mprof["apply32_count"]),
               "element_columns_per_cta_fp32": mm.get_shapes()[3],
               "gpu_launches": mlaunch}
        assert all(i["status"] == 0 for inf in minfos for i in inf)
        del mm
        return out

    mixed = pc32 = None
    if not args.no_mixed:
        mixed = precision_form(fnpf.FNPF_MIXED, args.mixed_cheb_degree)
        if pre == fnpf.FNPF_PMG:
            pc32 = precision_form(fnpf.FNPF_FP64_PC32, args.cheb_degree)

    # --- dominant kernel: the operator application inside the solves, timed live with
    #     CUDA events on the solve's stream over a further 3 RK4 steps
    mesh.profile_enable(True)
    for _ in range(3):
        flush.zero_()
        mesh.rk4_step(eta, phis, t, dt)
        t += dt
    torch.cuda.synchronize()
    prof = mesh.profile_read(reset=True)
    mesh.profile_enable(False)
    apply_ms = prof["apply_ms"] / max(1, prof["apply_count"])
    n = d["p"] + 1
    E = d["nx"] * d["ny"] * d["nz"]
    # algorithmic flops per application with the metric stored once per solve:
    # 6 one-dimensional contractions (12 n^4 per element) + G . grad u (18 n^3)
    flops = (12 * n ** 4 + 18 * n ** 3) * E
    achieved = flops / (apply_ms * 1e-3) / 1e12
    # dram bytes per application of the chosen kernel on this tank from one ncu capture of it
    # (shapes 3 and 4, the autotuner's picks here); none for other shapes or tanks
    bench_tank = n == 7 and d["nx"] == 32 and d["nz"] == 2
    traffic = {3: AXG_C2_DRAM_BYTES, 4: AXL_C2_DRAM_BYTES}.get(mesh.get_shapes()[0]) if bench_tank else None
    roofline = {"bound": "alu", "achieved": achieved, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                "frac": achieved / FP64_PEAK_TFLOPS, "traffic": traffic,
                "kernel": ("axg_kernel<double,7,3,C>" if mesh.get_shapes()[0] < 4 else
                           "axl_kernel<double,7,C,true>" if mesh.get_shapes()[0] < 8 else
                           "axz_kernel<double,7,C,2,true>")
                          + " + ring_gather (one FP64 operator application, stored metric), shape %d, C = %d"
                          % (mesh.get_shapes()[0], mesh.get_shapes()[2]),
                "flops_per_application": flops,
                "apply_ms": apply_ms, "applications": prof["apply_count"],
                "peak_note": "FP64 FMA peak derived from unit counts and max clock (152 SM x 2 DFMA/clk x "
                             "2070 MHz); the FP64 path is ALU-bound on GB300",
                "bytes_per_application": 2 * 8 * mesh.N + 6 * 8 * E * n ** 3,
                "hbm_frac_of_measured": (2 * 8 * mesh.N + 6 * 8 * E * n ** 3) / (apply_ms * 1e-3) / 1e9 / measured_hbm_gbs()}

    # --- adjoint (reverse mode, FP64, same mesh): K forward steps recording the tape (the
    #     recompute of a checkpointed gradient), the K taped reverse steps, and the adjoint
    #     that recomputes its step, each over the same sequence of states in reverse order
    adjoint = None
    if not args.no_adjoint and args.model == "fnpf":   # the adjoint is built for the nonlinear model
        K = max(2, args.steps // 2)

        def ev_pair():
            return torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

        states, fwd_t, rev_t, rec_t = [], [], [], []
        mesh.tape_begin(K)
        for k in range(K):
            states.append((eta.clone(), phis.clone(), t))
            flush.zero_()
            a_, b_ = ev_pair()
            a_.record(stream)
            mesh.rk4_step(eta, phis, t, dt)
            b_.record(stream)
            fwd_t.append((a_, b_))
            t += dt
        mesh.tape_end()
        le = torch.ones(mesh.ns, dtype=torch.float64, device=dev) / mesh.ns
        lp = torch.zeros_like(le)
        lh = torch.zeros_like(le)
        for k in reversed(range(K)):
            flush.zero_()
            a_, b_ = ev_pair()
            a_.record(stream)
            mesh.step_adjoint_taped(k, le, lp, le, lp, lh, dt)
            b_.record(stream)
            rev_t.append((a_, b_))
        le2 = torch.ones(mesh.ns, dtype=torch.float64, device=dev) / mesh.ns
        lp2, lh2 = torch.zeros_like(le2), torch.zeros_like(le2)
        for k in reversed(range(K)):
            es, ps, tk = states[k]
            flush.zero_()
            a_, b_ = ev_pair()
            a_.record(stream)
            mesh.step_adjoint(es, ps, le2, lp2, le2, lp2, lh2, tk, dt)
            b_.record(stream)
            rec_t.append((a_, b_))
        torch.cuda.synchronize()
        ms = lambda evs: statistics.mean(x.elapsed_time(y) for x, y in evs)
        fwd_step = total_ms / args.steps
        tape_ms, rev_ms, rec_ms = ms(fwd_t), ms(rev_t), ms(rec_t)
        grad_diff = float(torch.linalg.norm(le - le2) / torch.linalg.norm(le2))
        adjoint = {"ms_per_step": rev_ms, "ratio_to_forward": rev_ms / fwd_step,
                   "tape_forward_ms_per_step": tape_ms,
                   "checkpointed_ratio": (tape_ms + rev_ms) / fwd_step,
                   "recomputing_adjoint_ms_per_step": rec_ms, "recomputing_ratio": rec_ms / fwd_step,
                   "taped_vs_recomputing_rel_l2": grad_diff, "steps": K,
                   "note": "ratio_to_forward = taped adjoint (reverse) step / graph-replayed forward step; "
                           "checkpointed_ratio adds the forward recompute that records the tape (the cost per "
                           "step of a checkpointed gradient beyond its forward run); recomputing = "
                           "fnpf_step_adjoint, which re-solves the step itself"}

    # --- end to end through the public API: pinned host state in, step, state out
    eta_h = torch.empty(mesh.ns, dtype=torch.float64, pin_memory=True)
    phi_h = torch.empty(mesh.ns, dtype=torch.float64, pin_memory=True)
    eta_h.copy_(eta)
    phi_h.copy_(phis)
    e2e_ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(args.steps)]
    barrier()
    torch.cuda.synchronize()
    for k in range(args.steps):
        flush.zero_()
        e2e_ev[k][0].record(stream)
        eta.copy_(eta_h, non_blocking=True)
        phis.copy_(phi_h, non_blocking=True)
        mesh.rk4_step(eta, phis, t, dt)
        eta_h.copy_(eta, non_blocking=True)
        phi_h.copy_(phis, non_blocking=True)
        e2e_ev[k][1].record(stream)
        t += dt
    torch.cuda.synchronize()
    barrier()
    e2e_ms = sum(a.elapsed_time(b) for a, b in e2e_ev)
    e2e_ms = ranks.max(e2e_ms, dev)
    e2e = {"value": world * mesh.N * args.steps / (e2e_ms * 1e-3), "unit": UNIT,
           "h2d_bytes_per_step": 2 * 8 * mesh.ns, "d2h_bytes_per_step": 2 * 8 * mesh.ns}

    # --- measured FMA throughput (the ALU roofline's attainable peak), outside the timed region
    peaks = measure_fma_peaks(dev)
    roofline["peak_measured"] = peaks["fp64"]["tflops"]
    roofline["frac_of_measured_peak"] = roofline["achieved"] / peaks["fp64"]["tflops"]

    cpu = cpu_all = vs_oracle = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        host = host_cpu()
        sample_path = os.path.join(tempfile.gettempdir(), "fnpf_oracle_sample_%d.npz" % os.getpid())
        res = run_oracle_sample(8, 2, 0, out=sample_path)
        tot = sum(res["times"])
        cpu = {"value": res["N"] * len(res["times"]) / tot, "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": oracle_sample_desc(8, len(res["times"])), "host": host}
        procs = host["nproc"] or 1
        agg, n_s = run_oracle_replicas(8, 1, procs)
        cpu_all = {"value": agg, "unit": UNIT, "cores": procs, "kind": "oracle",
                   "sample": "%d copies of the oracle at once, one thread each, 1 RK4 step each of the 8x8x2 "
                             "sample tank (N=%d); aggregate over the slowest copy" % (procs, n_s), "host": host}
        # the GPU paths on the oracle's sample, from the same initial state, at the benchmark's rtol
        ref = np.load(sample_path)
        os.remove(sample_path)
        vs_oracle = {"sample": "8x8x2 elements, p=6, same seeded state, 2 RK4 steps; oracle solves to rtol 1e-14",
                     "rtol": args.rtol}
        ds = workload(8)
        hs = np.full((ds["p"] * 8) ** 2, ds["h0"])
        for name, prec_id, cheb in (("fp64", fnpf.FNPF_FP64, args.cheb_degree),
                                    ("mixed", fnpf.FNPF_MIXED, args.mixed_cheb_degree),
                                    ("fp64_pc32", fnpf.FNPF_FP64_PC32, args.cheb_degree)):
            if prec_id == fnpf.FNPF_FP64_PC32 and pre != fnpf.FNPF_PMG:
                continue
            so = fnpf.default_opts(precision=prec_id, rtol=args.rtol, max_iter=50000, precond=pre,
                                   cheb_degree=cheb, coarse_iters=args.coarse_degree,
                                   coarse_solver=coarse_mode(args), cheb_kind=args.cheb_kind,
                                   cheb_range=args.cheb_range, model=model_id(args), mg_schedule=schedule_id(args),
                                   projection=args.projection)
            sm = fnpf.Mesh(3, 8, 8, 2, ds["p"], True, True, hs, Lx=ds["Lx"], Ly=ds["Ly"], g=ds["g"], opts=so)
            sx, sy = sm.surface_coords()
            se0, sp0 = W.airy_plus_spectrum_state(ds, sx, sy, seed=2)
            se = torch.tensor(se0, dtype=torch.float64, device=dev)
            sp = torch.tensor(sp0, dtype=torch.float64, device=dev)
            sdt = W.period(ds["k"], ds["h0"], ds["g"]) / 100
            for k in range(2):
                sm.rk4_step(se, sp, k * sdt, sdt)
            torch.cuda.synchronize()
            ge, gp = se.cpu().numpy(), sp.cpu().numpy()
            vs_oracle[name] = {"eta": float(np.linalg.norm(ge - ref["eta"]) / np.linalg.norm(ref["eta"])),
                               "phis": float(np.linalg.norm(gp - ref["phis"]) / np.linalg.norm(ref["phis"]))}
            del sm
        if args.model != "fnpf":
            vs_oracle = None      # the oracle sample is the nonlinear model

    bar = None
    if rank == 0 and world == 1 and not args.no_bar:
        try:   # the mixed form's own configuration, shortened: 30 steps from rest, 5 timed after 3
            bar = bar_flume_run(args, 30, 5, 3)
        except Exception as e:   # reported in the line instead of ending the run
            bar = {"error": "%s: %s" % (type(e).__name__, str(e).splitlines()[0] if str(e) else "")}

    prism = None
    if rank == 0 and world == 1 and not args.no_prism:
        try:   # runs last: nothing measured above depends on it
            prism = prism_leg(dev, args, flush)
        except Exception as e:   # reported in the line instead of ending the run
            prism = {"error": "%s: %s" % (type(e).__name__, str(e).splitlines()[0] if str(e) else "")}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64" if args.precision == "fp64" else "f64+f32",
            "data": "synthetic",
            "config": {"workload": WORKLOAD, "dof": mesh.N, "surface_dof": mesh.ns, "precision": args.precision,
                       "precond": args.precond, "cheb_degree": cdeg, "coarse_degree": args.coarse_degree,
                       "coarse_solver": args.coarse_solver, "cheb_kind": args.cheb_kind,
                       "cheb_range": args.cheb_range, "model": args.model, "mg_schedule": args.mg_schedule,
                       "projection": args.projection,
                       "cta_shape": ("autotuned" if args.shape < 0 and not args.shapes else "forced"),
                       "element_columns_per_cta": mesh.get_shapes()[2],
                       "cta_shape_fp64": mesh.get_shapes()[0], "cta_shape_fp32": mesh.get_shapes()[1],
                       "headline_precision": args.precision, "l2": "flushed before every timed step (256 MB write, untimed)",
                       "parallelism": "replicas" if world > 1 else "single-gpu",
                       "cg_iters_per_solve_mean": statistics.mean(iters), "max_rel_res": rel_res,
                       "wall_s": wall},
            "roofline": roofline,
            "mixed": mixed, "fp64_pc32": pc32,
            "adjoint": adjoint,
            "rel_l2_vs_oracle": vs_oracle,
            "drift": drift,
            "fma_peaks_measured": peaks,
            "cpu_baseline": cpu,
            "cpu_baseline_all_cores": cpu_all,
            "e2e": e2e,
            "gpu_launches": launches,
            "clocks": clk.summary(),
            "bar": bar,
            "prism": prism,
        }
        print(json.dumps(line))
    ranks.close()
    return 0


PRISM_T0 = 4.0   # the flume runs from rest at t = 4 s: the generation ramp (5 T) is at 80 %


def prism_flume_run(dev, nx, ny, p, nz, steps, warm, rtol, precond, flush=None, precision=0, projection=0,
                    adjoint=False):
    """The prism path (operator, solve, w, projected conditions, RK4,
    relaxation zones) on the triangulated flume W.prism_flume from rest at
    t = 4 s: `warm` untimed steps, then `steps` steps timed with CUDA events on
    the current stream (L2 flushed before each when `flush` is given).
    Returns (state, ms per timed step, mean CG iterations per solve, mesh);
    with `adjoint`, also the mean time of fnpf_prism_step_adjoint over the
    same timed steps (the cotangent of sum(eta) at each step's start state)."""
    import torch

    from paper_2506_09435_gb300 import fnpf
    from paper_2506_09435_gb300 import workloads as W
    v, t, d = W.prism_flume(nx=nx, ny=ny, p=p, nz=nz)
    _, x, _ = fnpf.prism_numbering(v, t, d["p"])
    gm = fnpf.PrismMesh(v, t, d["p"], d["nz"])
    cr, gen = W.flume_zones(d, x)
    wv = W.flume_wave(d)
    gm.set_relaxation(cr, gen, wv["amp"], wv["kx"], wv["ky"], wv["omega"], wv["phase"], wv["ramp_time"])
    o = fnpf.PrismMesh.default_opts(rtol=rtol, g=d["g"], precond=precond, precision=precision, projection=projection)
    h = torch.full((gm.ns,), d["h0"], dtype=torch.float64, device=dev)
    eta = torch.zeros(gm.ns, dtype=torch.float64, device=dev)
    phis = torch.zeros(gm.ns, dtype=torch.float64, device=dev)
    dt = d["T"] / 40
    stream = torch.cuda.current_stream()
    iters, ms, ms_adj = [], 0.0, 0.0
    if adjoint:
        le, lz = torch.ones_like(eta), torch.zeros_like(eta)
        oe, op, oh = torch.empty_like(eta), torch.empty_like(eta), torch.empty_like(eta)
    for k in range(warm + steps):
        if flush is not None:
            flush.zero_()
        if adjoint and k >= warm:   # the adjoint of the step about to run, from the same start state
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            gm.step_adjoint(h, eta, phis, le, lz, oe, op, dt, lam_h=oh, opts=o, t=PRISM_T0 + k * dt)
            b.record(stream)
            torch.cuda.synchronize()
            ms_adj += a.elapsed_time(b)
            if flush is not None:
                flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        infos = gm.rk4_step(h, eta, phis, dt, o, t=PRISM_T0 + k * dt)
        b.record(stream)
        torch.cuda.synchronize()
        if k >= warm:
            ms += a.elapsed_time(b)
            iters += [i["iters"] for i in infos]
    out = ((eta, phis), ms / max(1, steps), statistics.mean(iters) if iters else 0.0, gm)
    return out + (ms_adj / max(1, steps),) if adjoint else out


def prism_operator_timing(dev, nx, ny, p, nz, reps=20):
    """The prism operator on the flume mesh: y = A(eta, h) x with the stored
    metric (the items of the solve: vertical derivatives, fluxes, vertical sums,
    node contractions, gather) and with the metric rebuilt per application
    (fnpf_prism_apply), each timed over `reps` applications with CUDA events;
    executed FP64 flops per prism 12 n nq nt + 18 n nq + 4 n^2 nt for the stored
    form (n = p + 1, nq = (p + 2)^2, nt = (p + 1)(p + 2) / 2)."""
    import torch

    from paper_2506_09435_gb300 import fnpf
    from paper_2506_09435_gb300 import workloads as W
    v, t, d = W.prism_flume(nx=nx, ny=ny, p=p, nz=nz)
    _, x_, y_ = fnpf.prism_numbering(v, t, p)
    gm = fnpf.PrismMesh(v, t, p, nz)
    xs = torch.tensor(x_, dtype=torch.float64, device=dev)
    eta = 0.01 * torch.cos(6.0 * xs)
    h = torch.full((gm.ns,), d["h0"], dtype=torch.float64, device=dev)
    x = torch.sin(torch.arange(gm.N, dtype=torch.float64, device=dev))
    y = torch.zeros(gm.N, dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream()
    n, nq, nt = p + 1, (p + 2) ** 2, (p + 1) * (p + 2) // 2
    prisms = 2 * nx * ny * nz
    out = {"prisms": prisms, "dof": gm.N, "reps": reps}

    def timed(fn):
        fn()   # first call: set-up
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        a.record(stream)
        for _ in range(reps):
            fn()
        b.record(stream)
        torch.cuda.synchronize()
        return 1e3 * a.elapsed_time(b) / reps

    # fnpf_prism_apply_stored rebuilds the metric and the diagonal before applying the operator;
    # fnpf_prism_diagonal is that rebuild alone, so the difference is the operator with the stored metric
    t_full = timed(lambda: gm.apply_stored(eta, h, x, y))
    t_geo = timed(lambda: gm.diagonal(eta, h, y))
    us = max(t_full - t_geo, 1e-3)
    flops = prisms * (12 * n * nq * nt + 18 * n * nq + 4 * n * n * nt)
    out["stored_metric"] = {"us_per_application": us, "us_metric_and_diagonal": t_geo,
                            "us_apply_stored_call": t_full, "flops_executed": flops, "gflops": flops / (us * 1e3),
                            "frac_of_fp64_peak": flops / (us * 1e-6) / (FP64_PEAK_TFLOPS * 1e12),
                            "applications_per_s": 1e6 / us}
    out["metric_per_application"] = {"us_per_application": timed(lambda: gm.apply(eta, h, x, y))}
    del gm
    return out


def prism_leg(dev, args, flush, size=(128, 32, 4, 2), sample=(6, 2, 3, 2, 2)):
    """Sub-object of the benchmark line: the prism path on the triangulated
    flume of `size` = (cells in x, cells in y, p, Nz) (throughput, CG
    iterations with the p-multigrid and with Jacobi), and its error against the
    oracle on the flume of `sample` = (cells in x, in y, p, Nz, RK4 steps)."""
    import numpy as np
    import torch

    from paper_2506_09435_gb300 import fnpf
    (nx, ny, p, nz), steps = size, max(1, min(args.steps, 5))
    (eta, phis), ms, it_pmg, gm = prism_flume_run(dev, nx, ny, p, nz, steps, 2, args.rtol, fnpf.FNPF_PMG, flush,
                                                  projection=8)
    out = {"workload": "prisms (Sec. 3.1.2) over a jittered triangulation of a walled 4 x 1 m flume, %d x %d cells "
                       "(%d triangles), Nz=%d, p=%d, h=0.4 m, generation and absorption zones, T = 1 s, dt = T/40, "
                       "from rest at t = 4 s" % (nx, ny, 2 * nx * ny, nz, p),
           "dof": gm.N, "surface_dof": gm.ns, "precond": "pmg", "projection": 8, "rtol": args.rtol, "steps": steps,
           "ms_per_step": ms, "value": gm.N / (ms * 1e-3), "unit": UNIT,
           "cg_iters_per_solve_mean": it_pmg, "finite": bool(torch.isfinite(eta).all())}
    del gm
    try:
        out["operator"] = prism_operator_timing(dev, nx, ny, p, nz)
    except Exception as e:
        out["operator"] = {"error": "%s: %s" % (type(e).__name__, str(e).splitlines()[0] if str(e) else "")}
    try:   # the step adjoint against the forward step (a fresh mesh: the same start states, 2 timed steps)
        _, ms_f, _, gm, ms_a = prism_flume_run(dev, nx, ny, p, nz, 2, 2, args.rtol, fnpf.FNPF_PMG, flush,
                                               projection=8, adjoint=True)
        out["adjoint"] = {"ms_per_step": ms_a, "forward_ms_per_step": ms_f, "ratio": ms_a / ms_f,
                          "note": "fnpf_prism_step_adjoint (forward stages recomputed) over fnpf_prism_rk4_step"}
        del gm
    except Exception as e:
        out["adjoint"] = {"error": "%s: %s" % (type(e).__name__, str(e).splitlines()[0] if str(e) else "")}
    try:   # FP64 defect correction around the FP32 PCG, from the same state for the same steps
        (em_, pm_), msm, itm, gm = prism_flume_run(dev, nx, ny, p, nz, steps, 2, args.rtol, fnpf.FNPF_PMG, flush,
                                                   precision=fnpf.FNPF_MIXED, projection=8)
        out["mixed"] = {"ms_per_step": msm, "value": gm.N / (msm * 1e-3), "inner_iters_per_solve_mean": itm,
                        "inner_rtol": 1e-5,
                        "rel_l2_vs_fp64": {"eta": float(torch.linalg.norm(em_ - eta) / torch.linalg.norm(eta)),
                                           "phis": float(torch.linalg.norm(pm_ - phis) / torch.linalg.norm(phis))}}
        del gm
    except Exception as e:
        out["mixed"] = {"error": "%s: %s" % (type(e).__name__, str(e).splitlines()[0] if str(e) else "")}
    try:   # the V-cycle in FP32 inside the FP64 PCG, from the same state for the same steps
        (e32, p32), ms32, it32, gm = prism_flume_run(dev, nx, ny, p, nz, steps, 2, args.rtol, fnpf.FNPF_PMG, flush,
                                                     precision=fnpf.FNPF_FP64_PC32, projection=8)
        out["fp64_pc32"] = {"ms_per_step": ms32, "value": gm.N / (ms32 * 1e-3), "cg_iters_per_solve_mean": it32,
                            "rel_l2_vs_fp64": {"eta": float(torch.linalg.norm(e32 - eta) / torch.linalg.norm(eta)),
                                               "phis": float(torch.linalg.norm(p32 - phis) / torch.linalg.norm(phis))}}
        del gm
    except Exception as e:
        out["fp64_pc32"] = {"error": "%s: %s" % (type(e).__name__, str(e).splitlines()[0] if str(e) else "")}
    try:
        _, ms_j, it_j, gm = prism_flume_run(dev, nx, ny, p, nz, 1, 2, args.rtol, fnpf.FNPF_JACOBI, flush)
        out["jacobi"] = {"ms_per_step": ms_j, "cg_iters_per_solve_mean": it_j}
        del gm
    except Exception as e:
        out["jacobi"] = {"error": "%s: %s" % (type(e).__name__, str(e).splitlines()[0] if str(e) else "")}
    if not args.no_cpu_baseline:
        try:
            _prism_vs_oracle(dev, sample, out)
        except Exception as e:
            out["rel_l2_vs_oracle"] = {"error": "%s: %s" % (type(e).__name__, str(e).splitlines()[0] if str(e) else "")}
    return out


def _prism_vs_oracle(dev, sample, out):
    """The oracle on the `sample` flume (a child process, one thread) and the
    GPU path from the same state: out["cpu_baseline"], out["rel_l2_vs_oracle"]."""
    import numpy as np

    from paper_2506_09435_gb300 import fnpf
    sx, sy, sp, snz, ssteps = sample
    path = os.path.join(tempfile.gettempdir(), "fnpf_prism_oracle_%d.npz" % os.getpid())
    code = PRISM_ORACLE_SAMPLE.format(root=ROOT, nx=sx, ny=sy, p=sp, nz=snz, t0=PRISM_T0, steps=ssteps, out=path)
    res = subprocess.run([sys.executable, "-c", code], env=dict(os.environ, **ONE_THREAD), capture_output=True,
                         text=True, check=True)
    rec = json.loads(res.stdout.strip().splitlines()[-1])
    ref = np.load(path)
    os.remove(path)
    (ge, gp), _, _, gm = prism_flume_run(dev, sx, sy, sp, snz, ssteps, 0, 1e-13, fnpf.FNPF_PMG)
    ge, gp = ge.cpu().numpy(), gp.cpu().numpy()
    out["cpu_baseline"] = {"value": rec["N"] * len(rec["times"]) / sum(rec["times"]), "unit": UNIT, "cores": 1,
                           "kind": "oracle",
                           "sample": "the same flume on %d x %d cells, p=%d, Nz=%d (N=%d), %d RK4 steps"
                                     % (sx, sy, sp, snz, rec["N"], ssteps)}
    out["rel_l2_vs_oracle"] = {"sample": out["cpu_baseline"]["sample"] + "; GPU rtol 1e-13, oracle direct solves",
                               "eta": float(np.linalg.norm(ge - ref["eta"]) / np.linalg.norm(ref["eta"])),
                               "phis": float(np.linalg.norm(gp - ref["phis"]) / np.linalg.norm(ref["phis"]))}
    del gm


def main_prism(args):
    """--mode prism: the prism leg of the step benchmark on its own."""
    import torch
    dev = torch.device("cuda", torch.cuda.current_device())
    with ClockSampler(dev.index) as clk:
        out = prism_leg(dev, args, None)
    out["clocks"] = clk.summary()
    print(json.dumps({"mode": "prism", **out}))
    return 0


def main_apply(args):
    """Laplacian applications per second on an nx x nx x nz periodic box of
    order p (FP64 operator, fnpf_apply), L2 flushed before every timed
    application; used for the operator roofline and its ncu captures."""
    import numpy as np
    import torch

    from paper_2506_09435_gb300 import fnpf
    from paper_2506_09435_gb300 import workloads as W

    d = W.periodic_box_3d(nx=args.nx, ny=args.nx, nz=args.nz, p=args.p, kh=2.0)
    ncx = d["p"] * d["nx"]
    mesh = fnpf.Mesh(3, d["nx"], d["ny"], d["nz"], d["p"], True, True, np.full(ncx * ncx, d["h0"]),
                     Lx=d["Lx"], Ly=d["Ly"], g=d["g"])
    x, y = mesh.surface_coords()
    eta0, _ = W.airy_plus_spectrum_state(d, x, y, seed=2)
    dev = torch.device("cuda", 0)
    if args.shape >= 0:
        mesh.set_shapes(args.shape, args.shape)
    else:                               # shapes timed for this mesh (fnpf_apply uses the on-the-fly metric)
        mesh.autotune(torch.tensor(eta0, dtype=torch.float64, device=dev))
    eta = torch.tensor(eta0, dtype=torch.float64, device=dev)
    gen = torch.Generator(device=dev)
    gen.manual_seed(5)
    xv = torch.randn(mesh.N, dtype=torch.float64, device=dev, generator=gen)
    yv = torch.empty_like(xv)
    apply = mesh.apply
    if args.precision == "mixed":      # the FP32 operator of the mixed path
        eta, xv, yv = eta.float(), xv.float(), yv.float()
        apply = mesh.apply_f32
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)
    for _ in range(args.warmup):
        apply(eta, xv, yv)
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    stream = torch.cuda.current_stream()
    for k in range(args.steps):
        flush.zero_()
        ev[k][0].record(stream)
        apply(eta, xv, yv)
        ev[k][1].record(stream)
    torch.cuda.synchronize()
    ms = statistics.mean(a.elapsed_time(b) for a, b in ev)
    n = d["p"] + 1
    E = d["nx"] * d["ny"] * d["nz"]
    flops = (12 * n ** 4 + 45 * n ** 3) * E      # on-the-fly metric: contractions + metric rebuild + G . grad u
    fp32 = args.precision == "mixed"
    tflops = flops / (ms * 1e-3) / 1e12
    gbs = (2 * xv.element_size() * mesh.N + 2 * xv.element_size() * mesh.ns) / (ms * 1e-3) / 1e9
    print(json.dumps({"mode": "apply", "precision": "fp32" if fp32 else "fp64",
                      "dof": mesh.N, "p": d["p"], "nx": d["nx"], "nz": d["nz"],
                      "element_columns_per_cta": mesh.get_shapes()[3 if fp32 else 2],
                      "ms_per_apply": ms, "applies_per_s": 1e3 / ms, "tflops_alg": tflops,
                      "frac_alu_peak": tflops / (FP32_PEAK_TFLOPS if fp32 else FP64_PEAK_TFLOPS),
                      "alu_peak_tflops": FP32_PEAK_TFLOPS if fp32 else FP64_PEAK_TFLOPS,
                      "gbs_alg": gbs, "frac_hbm_measured": gbs / measured_hbm_gbs(),
                      "l2": "flushed before every timed application"}))
    return 0


def main_ensemble(args):
    """Batched ensemble form: seeded independent periodic tanks (nx, ny in 8..96, 2
    layers, p in 3..7, kh in 0.5..3, steepness 0.01..0.06), FP32 operator and
    p-multigrid inside FP64 defect correction, each ensemble RK4 step one launch of
    a captured graph in which the tanks of each order share every kernel launch
    (batched groups); for comparison the same graph with one branch of per-tank
    kernels per tank (fork/join) and the tanks stepped one launch at a time.
    The working set (tens of millions of DOF) is far larger than L2, so no flush."""
    import numpy as np
    import torch

    from paper_2506_09435_gb300 import fnpf
    from paper_2506_09435_gb300 import workloads as W

    dev = torch.device("cuda", 0)
    tanks = W.ensemble_tanks(n=args.tanks, seed=5)
    opts = fnpf.default_opts(precision=fnpf.FNPF_MIXED, precond=fnpf.FNPF_PMG, rtol=args.rtol, inner_rtol=args.inner_rtol,
                             cheb_degree=args.mixed_cheb_degree, coarse_iters=args.coarse_degree,
                             coarse_solver=coarse_mode(args), cheb_kind=args.cheb_kind,
                             cheb_range=args.cheb_range, max_iter=50000, projection=args.projection)
    meshes, etas, phiss, dts, init = [], [], [], [], []
    for d in tanks:
        ncx, ncy = d["p"] * d["nx"], d["p"] * d["ny"]
        m = fnpf.Mesh(3, d["nx"], d["ny"], 2, d["p"], True, True, np.full(ncx * ncy, d["h0"]), Lx=d["Lx"],
                      Ly=d["Ly"], g=d["g"], opts=opts)
        if args.shape >= 0:
            m.set_shapes(args.shape, args.shape)
        x, y = m.surface_coords()
        e0, p0 = W.airy_plus_spectrum_state(d, x, y, seed=d["seed"], steepness=d["steepness"])
        meshes.append(m)
        init.append((e0, p0))
        etas.append(torch.tensor(e0, dtype=torch.float64, device=dev))
        phiss.append(torch.tensor(p0, dtype=torch.float64, device=dev))
        dts.append(W.period(d["k"], d["h0"], d["g"]) / 100)
    ndof = sum(m.N for m in meshes)
    ens = fnpf.Ensemble(meshes)
    stream = torch.cuda.current_stream()
    steps = [0] * len(meshes)
    for _ in range(max(2, args.warmup)):
        ens.rk4_step(etas, phiss, [k * dt for k, dt in zip(steps, dts)], dts)
        steps = [k + 1 for k in steps]
    torch.cuda.synchronize()
    n_warm = steps[0]
    for m in meshes:
        m.profile_read(reset=True)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    with ClockSampler(0) as clk:
        torch.cuda.synchronize()
        for k in range(args.steps):
            ev[k][0].record(stream)
            ens.rk4_step(etas, phiss, [s_ * dt for s_, dt in zip(steps, dts)], dts)
            ev[k][1].record(stream)
            steps = [s_ + 1 for s_ in steps]
        torch.cuda.synchronize()
    ens_ms = sum(a.elapsed_time(b) for a, b in ev)
    launches = sum(m.profile_read(reset=True)["launches"] for m in meshes)
    groups = ens.stats()
    # error of the batched mixed-precision states against the FP64 path: every tank
    # stepped in FP64 from the same initial state for the same steps, one at a time
    n_done = steps[0]
    err, err_tank, failures = [], [], []
    o64 = fnpf.default_opts(precond=fnpf.FNPF_PMG, rtol=args.rtol, max_iter=50000, projection=args.projection)
    for i, (d, (e0, p0), e_b, p_b, dt) in enumerate(zip(tanks, init, etas, phiss, dts)):
        ncx, ncy = d["p"] * d["nx"], d["p"] * d["ny"]
        m64 = fnpf.Mesh(3, d["nx"], d["ny"], 2, d["p"], True, True, np.full(ncx * ncy, d["h0"]), Lx=d["Lx"],
                        Ly=d["Ly"], g=d["g"], opts=o64)
        e64 = torch.tensor(e0, dtype=torch.float64, device=dev)
        p64 = torch.tensor(p0, dtype=torch.float64, device=dev)
        st = 0
        for k in range(n_done):
            st = m64.rk4_step(e64, p64, k * dt, dt, check=False)
            if st != 0:
                failures.append({"tank": i, "phase": "fp64 reference", "step": k, "status": st})
                break
        if st == 0:
            err.append(max(float(torch.linalg.norm(e_b - e64) / torch.linalg.norm(e64)),
                           float(torch.linalg.norm(p_b - p64) / torch.linalg.norm(p64))))
            err_tank.append(i)
        del m64
    torch.cuda.synchronize()
    # the same ensemble as one fork/join branch of per-tank kernels per tank
    ens.set_batching(False)
    ens.rk4_step(etas, phiss, [s_ * dt for s_, dt in zip(steps, dts)], dts)   # re-capture
    steps = [s_ + 1 for s_ in steps]
    for m in meshes:
        m.profile_read(reset=True)
    torch.cuda.synchronize()
    f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    f0.record(stream)
    for k in range(args.steps):
        ens.rk4_step(etas, phiss, [s_ * dt for s_, dt in zip(steps, dts)], dts)
        steps = [s_ + 1 for s_ in steps]
    f1.record(stream)
    torch.cuda.synchronize()
    fj_ms = f0.elapsed_time(f1)
    fj_launches = sum(m.profile_read(reset=True)["launches"] for m in meshes)
    ens.set_batching(True)
    # the same tanks, one launch (captured step graph) at a time
    for i, (m, e, p, dt, s_) in enumerate(zip(meshes, etas, phiss, dts, steps)):
        st = m.rk4_step(e, p, s_ * dt, dt, check=False)   # warm the single-tank graphs
        if st != 0:
            failures.append({"tank": i, "phase": "one at a time (first)", "step": s_, "status": st})
    steps = [s_ + 1 for s_ in steps]
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for k in range(args.steps):
        for i, (m, e, p, dt) in enumerate(zip(meshes, etas, phiss, dts)):
            st = m.rk4_step(e, p, steps[i] * dt, dt, check=False)
            if st != 0:
                failures.append({"tank": i, "phase": "one at a time", "step": steps[i], "status": st})
        steps = [s_ + 1 for s_ in steps]
    e1.record(stream)
    torch.cuda.synchronize()
    one_ms = e0.elapsed_time(e1)
    ok = all(bool(torch.isfinite(e).all()) for e in etas)
    print(json.dumps({
        "mode": "ensemble", "metric": "aggregate DOF·RK4-steps/s (batched ensemble)", "unit": UNIT,
        "value": ndof * args.steps / (ens_ms * 1e-3), "one_at_a_time": ndof * args.steps / (one_ms * 1e-3),
        "speedup_vs_one_at_a_time": one_ms / ens_ms, "tanks": len(meshes), "total_dof": ndof,
        "batched_groups": groups["groups"], "batched_tanks": groups["batched_tanks"],
        "fork_join": {"value": ndof * args.steps / (fj_ms * 1e-3), "ms_per_ensemble_step": fj_ms / args.steps,
                      "launches_per_ensemble_step": fj_launches / args.steps},
        "launch_reduction_vs_fork_join": fj_launches / max(1, launches),
        "ms_per_ensemble_step": ens_ms / args.steps, "steps": args.steps, "dtype": "f32 inner / f64 outer",
        "orders": sorted(set(d["p"] for d in tanks)), "finite": ok, "gpu_launches": launches,
        "launches_per_ensemble_step": launches / args.steps,
        "rel_l2_vs_fp64_path_max_over_tanks": max(err) if err else None, "steps_compared": n_done,
        "rel_l2_vs_fp64_path_worst": sorted(({"tank": i, "p": tanks[i]["p"], "nx": tanks[i]["nx"], "ny": tanks[i]["ny"],
                                              "kh": tanks[i]["k"] * tanks[i]["h0"], "steepness": tanks[i]["steepness"],
                                              "err": e} for i, e in zip(err_tank, err)),
                                            key=lambda r: -r["err"])[:3],
        "projection": args.projection, "failures": failures,
        "clocks": clk.summary(), "data": "synthetic"}))
    return 0


def schedule_id(args):
    return {"halve": 0, "two": 1, "step2": 2}[args.mg_schedule]


def model_id(args):
    from paper_2506_09435_gb300 import fnpf
    return fnpf.FNPF_LINEAR if args.model == "lpf" else fnpf.FNPF_NONLINEAR


def coarse_mode(args):
    from paper_2506_09435_gb300 import fnpf
    return fnpf.FNPF_COARSE_CLUSTER if args.coarse_solver == "cluster" else fnpf.FNPF_COARSE_LAUNCHES


def main_convergence(args):
    """Accuracy study on a steady nonlinear wave (the paper's nonlinear
    convergence tests, Sec. 4): a stream-function wave of steepness H/L = 0.05
    at kh = 1 in a periodic 2D tank of one wavelength, 2 vertical elements,
    carried for one period (dt = T/128); max-norm errors of eta (over H) and
    of phi_eta (relative) against the exact travelling wave, for p = 3..8 at
    4 elements per wavelength and for 2..16 elements at p = 4."""
    import numpy as np
    import torch

    from paper_2506_09435_gb300 import fnpf
    from paper_2506_09435_gb300 import workloads as W

    def run(p, nx, nsteps=128):
        d, wave = W.stream_function_tank_2d(nx=nx, nz=2, p=p, steepness=0.05)
        gm = fnpf.Mesh(2, nx, 1, 2, p, True, False, np.full(p * nx, d["h0"]), Lx=d["Lx"], g=d["g"],
                       opts=fnpf.default_opts(rtol=1e-13, max_iter=50000, precond=fnpf.FNPF_PMG))
        x, _ = gm.surface_coords()
        dev = torch.device("cuda:0")
        eta = torch.tensor(wave.eta(x), dtype=torch.float64, device=dev)
        phis = torch.tensor(wave.phis(x), dtype=torch.float64, device=dev)
        T = wave.period()
        for n in range(nsteps):
            gm.rk4_step(eta, phis, n * T / nsteps, T / nsteps)
        torch.cuda.synchronize()
        ref = wave.phis(x, T)
        return {"p": p, "nx": nx, "dof": gm.N,
                "err_eta_over_H": float(np.max(np.abs(eta.cpu().numpy() - wave.eta(x, T))) / wave.H),
                "err_phi_rel": float(np.max(np.abs(phis.cpu().numpy() - ref)) / np.max(np.abs(ref)))}

    rows = [run(p, 4) for p in range(3, 9)] + [run(4, nx) for nx in (2, 8, 16)]
    print(json.dumps({"mode": "convergence", "wave": "stream function, kh = 1, H/L = 0.05, one period, dt = T/128",
                      "rows": rows}))
    return 0


def main_bar(args):
    """--mode bar: bar_flume_run for `--bar-steps` steps, `--steps` timed after `--warmup`."""
    out = bar_flume_run(args, args.bar_steps, args.steps, args.warmup)
    print(json.dumps({"mode": "bar", **out}))
    return 0


def bar_flume_run(args, bar_steps, steps, warmup):
    """The submerged-bar flume (256 x 16 x 3 elements, p = 5, 1,660,176 DOF,
    walls, variable depth; incident T = 2.02 s, H = 0.02 m through a
    generation zone, absorption zone at the outlet), run from rest for
    `bar_steps` RK4 steps of dt = T/100 in FP64, in the defect-correction
    mixed form and in FP64 PCG with the FP32 p-multigrid preconditioner.
    Throughput from `steps` timed steps after `warmup`; accuracy of each
    mixed form against the FP64 run at 8 probes spread over x = 8 ... 30 m at
    y = 0.5 m (the nearest surface node) and over the whole surface."""
    import numpy as np
    import torch

    from paper_2506_09435_gb300 import fnpf
    from paper_2506_09435_gb300 import workloads as W

    d = W.bar_flume()
    dims = (3, d["nx"], d["ny"], d["nz"], d["p"], False, False)
    ncx = d["p"] * d["nx"] + 1
    ncy = d["p"] * d["ny"] + 1
    probe = fnpf.Mesh(*dims, np.full(ncx * ncy, d["h0"]), Lx=d["Lx"], Ly=d["Ly"], g=d["g"])
    x, y = probe.surface_coords()
    del probe
    h = W.bar_depth(x)
    cr, gen = W.flume_zones(d, x)
    wave = W.flume_wave(d)
    px = np.linspace(8.0, 30.0, 8)
    pcols = [int(np.argmin((x - xp) ** 2 + (y - 0.5) ** 2)) for xp in px]
    dt = d["T"] / 100
    dev = torch.device("cuda", 0)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()
    rows, ref = [], None
    for name, prec in (("fp64", fnpf.FNPF_FP64), ("mixed", fnpf.FNPF_MIXED), ("pc32", fnpf.FNPF_FP64_PC32)):
        opts = fnpf.default_opts(precision=prec, precond=fnpf.FNPF_PMG, rtol=args.rtol, inner_rtol=args.inner_rtol,
                                 max_iter=50000, cheb_degree=args.cheb_degree, coarse_iters=args.coarse_degree)
        gm = fnpf.Mesh(*dims, h, Lx=d["Lx"], Ly=d["Ly"], g=d["g"], opts=opts)
        gm.set_relaxation(cr, gen, **wave)
        eta = torch.zeros(gm.ns, dtype=torch.float64, device=dev)
        phis = torch.zeros_like(eta)
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(steps)]
        iters = []
        for n in range(max(bar_steps, warmup + steps)):
            k = n - warmup
            timed = 0 <= k < steps
            if timed:
                flush.zero_()
                ev[k][0].record(stream)
            inf = gm.rk4_step(eta, phis, n * dt, dt, info=timed)
            if timed:
                ev[k][1].record(stream)
                iters += [i["iters"] for i in inf]
        torch.cuda.synchronize()
        ms = sum(a.elapsed_time(b) for a, b in ev) / steps
        e = eta.cpu().numpy()
        row = {"precision": name, "value": gm.N / (ms * 1e-3), "unit": UNIT, "ms_per_step": ms,
               "cg_iters_per_solve_mean": statistics.mean(iters)}
        if ref is None:
            ref = e
            row["probe_eta_max"] = float(np.max(np.abs(e[pcols])))
        else:
            row["probe_rel_err_vs_fp64"] = float(np.max(np.abs(e[pcols] - ref[pcols])) / np.max(np.abs(ref[pcols])))
            row["field_rel_l2_vs_fp64"] = float(np.linalg.norm(e - ref) / np.linalg.norm(ref))
        rows.append(row)
        del gm
    return {"workload": "submerged-bar flume 256x16x3, p=5, walls, relaxation zones",
            "dof": ncx * ncy * (d["p"] * d["nz"] + 1), "steps_run": max(bar_steps, warmup + steps),
            "timed_steps": steps, "warmup": warmup, "dt": dt, "probes_x": px.tolist(), "rows": rows,
            "data": "synthetic"}


def main_cylinder(args):
    """Adjoint form on the cylinder O-grid (64 azimuthal x 24 radial x 3
    elements, p = 4, isoparametric, 322,816 DOF; ka = kh = 1, outer radius 10a
    with a sponge ring over 0.8 R .. R; linear incident wave of steepness
    0.01, dt = T/64), FP64 p-multigrid: the forward RK4 step, the hand-written
    adjoint step, and a checkpointed gradient (checkpoints every 16 steps)
    through the torch.autograd.Function of 2 x 16 steps."""
    import numpy as np
    import torch

    from paper_2506_09435_gb300 import fnpf
    from paper_2506_09435_gb300 import workloads as W
    from paper_2506_09435_gb300.autograd import rk4_run

    d = W.cylinder_case()
    dims = (3, d["nx"], d["ny"], d["nz"], d["p"], True, False)
    ncx, ncy = d["p"] * d["nx"], d["p"] * d["ny"] + 1
    box = fnpf.Mesh(*dims, np.full(ncx * ncy, d["h0"]), Lx=d["Lx"], Ly=d["Ly"], g=d["g"])
    th, sr = box.surface_coords()
    del box
    X, Y = W.ogrid_map(th, sr, a=d["a"], R=d["R"])
    h = np.full(X.size, d["h0"])
    opts = fnpf.default_opts(precond=fnpf.FNPF_PMG, rtol=args.rtol, max_iter=50000, cheb_degree=args.cheb_degree,
                             coarse_iters=args.coarse_degree)
    mesh = fnpf.Mesh(*dims, h, X=X, Y=Y, g=d["g"], opts=opts)
    r = np.hypot(X, Y)
    cr = np.where(r >= 0.8 * d["R"], W.relaxation_weight((d["R"] - r) / (0.2 * d["R"])), 0.0)
    om = 2 * np.pi / d["T"]
    mesh.set_relaxation(cr, np.zeros_like(cr), amp=0.0, kx=d["k"], omega=om, ramp_time=5 * d["T"])
    amp = 0.5 * 0.01 * 2 * np.pi / d["k"]
    eta0 = amp * np.cos(d["k"] * X)
    phi0 = d["g"] * amp / om * np.cosh(d["k"] * (eta0 + h)) / np.cosh(d["k"] * h) * np.sin(d["k"] * X)
    dev = torch.device("cuda", 0)
    eta = torch.tensor(eta0, dtype=torch.float64, device=dev)
    phis = torch.tensor(phi0, dtype=torch.float64, device=dev)
    dt = d["T"] / 64
    stream = torch.cuda.current_stream()
    t = 0.0
    for _ in range(args.warmup):
        mesh.rk4_step(eta, phis, t, dt)
        t += dt
    torch.cuda.synchronize()

    def timed(fn, k):
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(k)]
        for a_, b_ in ev:
            a_.record(stream)
            fn()
            b_.record(stream)
        torch.cuda.synchronize()
        return statistics.mean(a_.elapsed_time(b_) for a_, b_ in ev)

    fwd_ms = timed(lambda: mesh.rk4_step(eta, phis, t, dt), args.steps)
    # adjoint steps over a sequence of states in reverse order (as in a gradient): K forward
    # steps recording the tape, then the K taped reverse steps
    K = max(2, args.steps // 2)
    mesh.tape_begin(K)
    tape_ms = timed(lambda: mesh.rk4_step(eta, phis, t, dt), K)
    mesh.tape_end()
    le = torch.ones(mesh.ns, dtype=torch.float64, device=dev) / mesh.ns
    lp = torch.zeros_like(le)
    lh = torch.zeros_like(le)
    slots = list(reversed(range(K)))
    adj_ms = timed(lambda: mesh.step_adjoint_taped(slots.pop(0), le, lp, le, lp, lh, dt), K)
    # checkpointed gradient of J = sum eta_N^2 over 32 steps, checkpoints every 16
    e0 = eta.detach().clone().requires_grad_(True)
    p0 = phis.detach().clone().requires_grad_(True)
    ht = torch.tensor(h, dtype=torch.float64, device=dev, requires_grad=True)
    torch.cuda.synchronize()
    w0 = time.perf_counter()
    eN, pN = rk4_run(mesh, e0, p0, ht, t, dt, 32, every=16)
    torch.cuda.synchronize()
    w1 = time.perf_counter()
    (eN * eN).sum().backward()
    torch.cuda.synchronize()
    w2 = time.perf_counter()
    finite = bool(torch.isfinite(e0.grad).all() and torch.isfinite(p0.grad).all() and torch.isfinite(ht.grad).all())
    # the configuration's objective: J = int F_x dt (horizontal force on the cylinder)
    # over steps 16..32, gradient with respect to the initial state and the depth
    from paper_2506_09435_gb300.objectives import WallForce, cylinder_force_objective
    wf = WallForce(mesh, X, Y, Mz=d["p"] + 2)
    f0 = eta.detach().clone().requires_grad_(True)
    q0 = phis.detach().clone().requires_grad_(True)
    hf = torch.tensor(h, dtype=torch.float64, device=dev, requires_grad=True)
    torch.cuda.synchronize()
    v0 = time.perf_counter()
    Jf = cylinder_force_objective(mesh, wf, f0, q0, hf, t, dt, 16, 32, every=16)
    torch.cuda.synchronize()
    v1 = time.perf_counter()
    Jf.backward()
    torch.cuda.synchronize()
    v2 = time.perf_counter()
    force = {"objective": "J = int F_x dt over steps 16..32 (force on the cylinder, still-water wetted surface)",
             "J": float(Jf.detach()), "forward_s": v1 - v0, "backward_s": v2 - v1, "ratio": (v2 - v1) / (v1 - v0),
             "grad_norm_eta0": float(torch.linalg.norm(f0.grad)), "grad_norm_h": float(torch.linalg.norm(hf.grad)),
             "finite": bool(torch.isfinite(f0.grad).all() and torch.isfinite(hf.grad).all())}
    print(json.dumps({"mode": "cylinder", "workload": "cylinder O-grid 64x24x3, p=4, ka=kh=1, R=10a, sponge ring",
                      "dof": mesh.N, "forward_ms_per_step": fwd_ms, "adjoint_ms_per_step": adj_ms,
                      "tape_forward_ms_per_step": tape_ms,
                      "adjoint_ratio_to_forward": (tape_ms + adj_ms) / fwd_ms,
                      "checkpointed_gradient": {"steps": 32, "every": 16, "forward_s": w1 - w0,
                                                "backward_s": w2 - w1, "ratio": (w2 - w1) / (w1 - w0),
                                                "finite": finite},
                      "force_gradient": force,
                      "data": "synthetic"}))
    return 0


def main_peaks(args):
    """Measured FP64 and FP32 FMA throughput of this GPU (fnpf_fma_probe),
    with the SM clocks sampled while the probes run."""
    import torch
    dev = torch.device("cuda", 0)
    with ClockSampler(0) as clk:
        peaks = measure_fma_peaks(dev, reps=20)
    derived = {"fp64": FP64_PEAK_TFLOPS, "fp32": FP32_PEAK_TFLOPS}
    for k in peaks:
        peaks[k]["derived_tflops"] = derived[k]
        peaks[k]["frac_of_derived"] = peaks[k]["tflops"] / derived[k]
    print(json.dumps({"mode": "peaks", "fma": peaks, "clocks": clk.summary(),
                      "how": "8 independent FMA chains per thread, 152 x 16 CTAs of 256 threads, best of 20 "
                             "launches timed with CUDA events; derived = 152 SM x FMA/clk x 2 flop x 2070 MHz"}))
    return 0


def main():
    args = parse()
    if args.mode == "peaks":
        return main_peaks(args)
    if args.mode == "convergence":
        return main_convergence(args)
    if args.mode == "bar":
        return main_bar(args)
    if args.mode == "cylinder":
        return main_cylinder(args)
    if args.mode == "ensemble":
        return main_ensemble(args)
    if args.mode == "prism":
        return main_prism(args)
    if args.impl == "reference":
        return main_reference(args)
    if args.mode == "apply":
        return main_apply(args)
    return main_gb300(args)


if __name__ == "__main__":
    sys.exit(main())
