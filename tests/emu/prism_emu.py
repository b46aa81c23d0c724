"""Build and call the host harness of the prism solve and step
(tests/emu/prism_step_host.cpp): the library's kernel bodies and orchestration
(paper_2506_09435_gb300/csrc/prism_step.h) compiled as plain C++ and run item
by item on host arrays.  Tests only."""
import ctypes
import os
import shutil
import subprocess

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
PKG = os.path.join(ROOT, "paper_2506_09435_gb300")


def asan_runtime():
    """Path of the AddressSanitizer runtime of g++, or None."""
    cxx = shutil.which("g++")
    if not cxx:
        return None
    r = subprocess.run([cxx, "-print-file-name=libasan.so"], capture_output=True, text=True)
    path = r.stdout.strip()
    return path if r.returncode == 0 and os.path.isabs(path) and os.path.exists(path) else None


def build(out_dir, asan=False):
    """Compiles the harness against the in-tree libfnpf.so (its host
    functions: numbering, tables); returns the path of the shared object."""
    from paper_2506_09435_gb300 import build as B
    B.build()
    out = os.path.join(out_dir, "libprism_emu%s.so" % ("_asan" if asan else ""))
    cmd = ["g++", "-std=c++17", "-shared", "-fPIC", "-Wall", "-Werror",
           "-I" + os.path.join(ROOT, "include"), "-I" + os.path.join(PKG, "csrc"),
           os.path.join(HERE, "prism_step_host.cpp"), "-L" + PKG, "-l:libfnpf.so", "-Wl,-rpath," + PKG, "-o", out]
    cmd[1:1] = ["-O1", "-g", "-fsanitize=address", "-fno-omit-frame-pointer"] if asan else ["-O2"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("harness build failed:\n" + r.stdout + r.stderr)
    return out


class PrismOpts(ctypes.Structure):
    _fields_ = [("rtol", ctypes.c_double), ("max_iter", ctypes.c_int), ("mass_rtol", ctypes.c_double),
                ("mass_max_iter", ctypes.c_int), ("g", ctypes.c_double), ("model", ctypes.c_int),
                ("precond", ctypes.c_int), ("cheb_degree", ctypes.c_int), ("coarse_iters", ctypes.c_int),
                ("cheb_range", ctypes.c_double), ("precision", ctypes.c_int), ("projection", ctypes.c_int),
                ("inner_rtol", ctypes.c_double), ("max_outer", ctypes.c_int)]


def opts(rtol=1e-10, max_iter=20000, mass_rtol=1e-13, g=9.81, linear=False, pmg=False, cheb_degree=3,
         coarse_iters=6, cheb_range=40.0, pc32=False, projection=0, mixed=False, inner_rtol=1e-5, max_outer=20):
    return PrismOpts(rtol, max_iter, mass_rtol, 5000, g, int(linear), int(pmg), cheb_degree, coarse_iters,
                     cheb_range, 1 if mixed else (2 if pc32 else 0), projection, inner_rtol, max_outer)


class SolveInfo(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int), ("outer_iters", ctypes.c_int), ("rel_res", ctypes.c_double),
                ("status", ctypes.c_int), ("ms", ctypes.c_float)]


def _p(a):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(ctypes.c_void_p)


class Harness:
    def __init__(self, path):
        vp = ctypes.c_void_p
        lib = ctypes.CDLL(path)
        lib.emu_create.restype = vp
        lib.emu_create.argtypes = [vp, ctypes.c_int, vp, ctypes.c_int, ctypes.c_int, ctypes.c_int]
        lib.emu_destroy.argtypes = [vp]
        lib.emu_destroy.restype = None
        lib.emu_sizes.argtypes = [vp] + [ctypes.POINTER(ctypes.c_int64)] * 3
        lib.emu_sizes.restype = None
        sig = {"emu_diagonal": [vp] * 4, "emu_apply_stored": [vp] * 5, "emu_apply_items": [vp] * 5, "emu_laplace_solve": [vp] * 7, "emu_precond_apply": [vp] * 6,
               "emu_laplace_solve_vjp": [vp] * 9,
               "emu_step_adjoint": [vp] * 10 + [ctypes.c_double, ctypes.c_double],
               "emu_dtn": [vp] * 7, "emu_rhs": [vp] * 8, "emu_rk4_step": [vp] * 5 + [ctypes.c_double, ctypes.c_double, vp],
               "emu_set_relaxation": [vp] * 3 + [ctypes.c_double] * 6, "emu_invariants": [vp] * 7}
        sig["emu_set_filter"] = [vp, ctypes.c_double, ctypes.c_int, ctypes.c_int]
        sig["emu_filter_apply"] = [vp, vp]
        for nm, args in sig.items():
            getattr(lib, nm).argtypes = args
            getattr(lib, nm).restype = ctypes.c_int
        self.lib = lib

    def mesh(self, verts, tris, p, nz):
        return EmuMesh(self.lib, verts, tris, p, nz)


class EmuMesh:
    def __init__(self, lib, verts, tris, p, nz):
        v = np.ascontiguousarray(verts, dtype=np.float64)
        t = np.ascontiguousarray(tris, dtype=np.int32)
        self.lib = lib
        self.h = lib.emu_create(_p(v), len(v), t.ctypes.data_as(ctypes.c_void_p), len(t), int(p), int(nz))
        if not self.h:
            raise ValueError("bad prism mesh")
        N, ns, _ = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
        lib.emu_sizes(self.h, ctypes.byref(N), ctypes.byref(ns), ctypes.byref(_))
        self.N, self.ns = N.value, ns.value

    def __del__(self):
        if getattr(self, "h", None):
            self.lib.emu_destroy(self.h)
            self.h = None

    def launches(self):
        N, ns, n = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
        self.lib.emu_sizes(self.h, ctypes.byref(N), ctypes.byref(ns), ctypes.byref(n))
        return n.value

    def diagonal(self, eta, h):
        d = np.zeros(self.N)
        assert self.lib.emu_diagonal(self.h, _p(eta), _p(h), _p(d)) == 0
        return d

    def apply_stored(self, eta, h, x):
        y = np.zeros(self.N)
        assert self.lib.emu_apply_stored(self.h, _p(eta), _p(h), _p(x), _p(y)) == 0
        return y

    def apply_items(self, eta, h, x):
        y = np.zeros(self.N)
        assert self.lib.emu_apply_items(self.h, _p(eta), _p(h), _p(x), _p(y)) == 0
        return y

    def laplace_solve(self, opts, eta, h, phis, phi):
        info = SolveInfo()
        st = self.lib.emu_laplace_solve(self.h, ctypes.byref(opts), _p(eta), _p(h), _p(phis), _p(phi),
                                        ctypes.byref(info))
        return st, info

    def precond_apply(self, opts, eta, h, r):
        z = np.zeros(self.N)
        st = self.lib.emu_precond_apply(self.h, ctypes.byref(opts), _p(eta), _p(h), _p(r), _p(z))
        assert st == 0, st
        return z

    def laplace_solve_vjp(self, opts, eta, h, phi, lam):
        le, lp, lh = np.zeros(self.ns), np.zeros(self.ns), np.zeros(self.ns)
        st = self.lib.emu_laplace_solve_vjp(self.h, ctypes.byref(opts), _p(eta), _p(h), _p(phi), _p(lam), _p(le),
                                            _p(lp), _p(lh))
        assert st == 0, st
        return le, lp, lh

    def step_adjoint(self, opts, h, eta, phis, lam_e, lam_p, dt, t=0.0):
        oe, op, oh = np.zeros(self.ns), np.zeros(self.ns), np.zeros(self.ns)
        st = self.lib.emu_step_adjoint(self.h, ctypes.byref(opts), _p(h), _p(eta), _p(phis), _p(lam_e), _p(lam_p),
                                       _p(oe), _p(op), _p(oh), float(t), float(dt))
        return st, oe, op, oh

    def dtn(self, opts, eta, h, phis):
        w, info = np.zeros(self.ns), SolveInfo()
        st = self.lib.emu_dtn(self.h, ctypes.byref(opts), _p(eta), _p(h), _p(phis), _p(w), ctypes.byref(info))
        return st, w

    def rhs(self, opts, eta, h, phis):
        ke, kp, info = np.zeros(self.ns), np.zeros(self.ns), SolveInfo()
        st = self.lib.emu_rhs(self.h, ctypes.byref(opts), _p(eta), _p(h), _p(phis), _p(ke), _p(kp),
                              ctypes.byref(info))
        return st, ke, kp

    def set_filter(self, alpha, order=2, cutoff=0):
        assert self.lib.emu_set_filter(self.h, float(alpha), int(order), int(cutoff)) == 0

    def filter_apply(self, f):
        out = np.array(f, dtype=np.float64, copy=True)
        assert self.lib.emu_filter_apply(self.h, _p(out)) == 0
        return out

    def invariants(self, opts, eta, h, phis):
        M, En = ctypes.c_double(), ctypes.c_double()
        assert self.lib.emu_invariants(self.h, ctypes.byref(opts), _p(eta), _p(h), _p(phis), ctypes.byref(M),
                                       ctypes.byref(En)) == 0
        return M.value, En.value

    def set_relaxation(self, cr, gen, amp, kx, ky, omega, phase, ramp_time):
        self._cr, self._gen = np.ascontiguousarray(cr, dtype=np.float64), np.ascontiguousarray(gen, dtype=np.float64)
        assert self.lib.emu_set_relaxation(self.h, _p(self._cr), _p(self._gen), amp, kx, ky, omega, phase,
                                           ramp_time) == 0

    def rk4_step(self, opts, h, eta, phis, dt, t=0.0):
        infos = (SolveInfo * 4)()
        st = self.lib.emu_rk4_step(self.h, ctypes.byref(opts), _p(h), _p(eta), _p(phis), float(t), float(dt),
                                   infos)
        return st, [infos[i].iters for i in range(4)]
