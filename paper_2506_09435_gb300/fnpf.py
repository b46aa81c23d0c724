"""Python binding of the C ABI in include/fnpf.h (argument marshalling only).

Every computation runs in libfnpf.so's CUDA kernels; this module only turns
torch tensors into device pointers and streams into cudaStream_t handles.
Importing it fails loudly when the shared library is missing: there is no
CPU fallback.
"""
import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libfnpf.so")

FNPF_OK, FNPF_EINVAL, FNPF_ENOMEM, FNPF_ECUDA, FNPF_ENOCONV, FNPF_EBREAKDOWN, FNPF_EDIVERGED, \
    FNPF_EUNSUPPORTED = range(8)
FNPF_BOX, FNPF_ISOPARAMETRIC = 0, 1
FNPF_FP64, FNPF_MIXED = 0, 1
FNPF_JACOBI, FNPF_PMG = 0, 1
FNPF_FP64_PC32 = 2
FNPF_COARSE_LAUNCHES, FNPF_COARSE_CLUSTER = 0, 1
FNPF_CHEB_FIRST, FNPF_CHEB_FOURTH = 1, 4
FNPF_NONLINEAR, FNPF_LINEAR = 0, 1
FNPF_MG_HALVE, FNPF_MG_TWO_LEVEL, FNPF_MG_STEP2 = 0, 1, 2

_dp = ctypes.POINTER(ctypes.c_double)


class MeshDesc(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int), ("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
                ("p", ctypes.c_int), ("periodic_x", ctypes.c_int), ("periodic_y", ctypes.c_int),
                ("horiz_kind", ctypes.c_int), ("Lx", ctypes.c_double), ("Ly", ctypes.c_double),
                ("X", _dp), ("Y", _dp), ("h", _dp), ("g", ctypes.c_double)]


class Opts(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int), ("precond", ctypes.c_int), ("rtol", ctypes.c_double),
                ("atol", ctypes.c_double), ("max_iter", ctypes.c_int), ("check_every", ctypes.c_int),
                ("cheb_degree", ctypes.c_int), ("coarse_iters", ctypes.c_int), ("inner_rtol", ctypes.c_double),
                ("max_outer", ctypes.c_int), ("use_graphs", ctypes.c_int), ("store_metric", ctypes.c_int),
                ("coarse_solver", ctypes.c_int), ("cheb_kind", ctypes.c_int), ("cheb_range", ctypes.c_double),
                ("model", ctypes.c_int), ("mg_schedule", ctypes.c_int), ("projection", ctypes.c_int)]


class PrismOpts(ctypes.Structure):
    _fields_ = [("rtol", ctypes.c_double), ("max_iter", ctypes.c_int), ("mass_rtol", ctypes.c_double),
                ("mass_max_iter", ctypes.c_int), ("g", ctypes.c_double), ("model", ctypes.c_int),
                ("precond", ctypes.c_int), ("cheb_degree", ctypes.c_int), ("coarse_iters", ctypes.c_int),
                ("cheb_range", ctypes.c_double), ("precision", ctypes.c_int), ("projection", ctypes.c_int),
                ("inner_rtol", ctypes.c_double), ("max_outer", ctypes.c_int)]


class SolveInfo(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int), ("outer_iters", ctypes.c_int), ("rel_res", ctypes.c_double),
                ("status", ctypes.c_int), ("ms", ctypes.c_float)]

    def as_dict(self):
        return dict(iters=self.iters, outer_iters=self.outer_iters, rel_res=self.rel_res, status=self.status,
                    ms=self.ms)


class Filter(ctypes.Structure):
    _fields_ = [("alpha", ctypes.c_double), ("order", ctypes.c_int), ("cutoff", ctypes.c_int)]


class Relaxation(ctypes.Structure):
    _fields_ = [("cr", _dp), ("gen", _dp), ("amp", ctypes.c_double), ("kx", ctypes.c_double),
                ("ky", ctypes.c_double), ("omega", ctypes.c_double), ("phase", ctypes.c_double),
                ("ramp_time", ctypes.c_double)]


def load():
    if not os.path.exists(LIB_PATH):
        raise RuntimeError("libfnpf.so is not built (run __graft_entry__.build() or "
                           "python -m paper_2506_09435_gb300.build); there is no CPU fallback")
    lib = ctypes.CDLL(LIB_PATH)
    vp, i64p = ctypes.c_void_p, ctypes.POINTER(ctypes.c_int64)
    sig = {
        "fnpf_count_dofs": [ctypes.POINTER(MeshDesc), i64p, i64p],
        "fnpf_create_mesh": [ctypes.POINTER(MeshDesc), ctypes.POINTER(Opts), ctypes.POINTER(vp)],
        "fnpf_set_opts": [vp, ctypes.POINTER(Opts)],
        "fnpf_mesh_sizes": [vp, i64p, i64p],
        "fnpf_surface_coords": [vp, _dp, _dp],
        "fnpf_apply": [vp, vp, vp, vp, vp],
        "fnpf_diagonal": [vp, vp, vp, vp],
        "fnpf_precond_apply": [vp, vp, vp, vp, vp],
        "fnpf_set_filter": [vp, ctypes.POINTER(Filter)],
        "fnpf_set_dealias": [vp, ctypes.c_int],
        "fnpf_filter_apply": [vp, vp, vp],
        "fnpf_apply_f32": [vp, vp, vp, vp, vp],
        "fnpf_laplace_solve": [vp, vp, vp, vp, ctypes.POINTER(SolveInfo), vp],
        "fnpf_dtn": [vp, vp, vp, vp, ctypes.POINTER(SolveInfo), vp],
        "fnpf_zakharov_rhs": [vp, vp, vp, vp, vp, vp, vp],
        "fnpf_rk4_step": [vp, vp, vp, ctypes.c_double, ctypes.c_double, ctypes.POINTER(SolveInfo), vp],
        "fnpf_apply_noalloc": [ctypes.POINTER(MeshDesc), vp, vp, vp, vp, vp],
        "fnpf_invariants": [vp, vp, vp, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double),
                            ctypes.POINTER(SolveInfo), vp],
        "fnpf_fma_probe": [ctypes.c_int, ctypes.c_int, ctypes.c_int, vp, ctypes.POINTER(ctypes.c_double), vp],
        "fnpf_set_relaxation": [vp, ctypes.POINTER(Relaxation)],
        "fnpf_step_adjoint": [vp, vp, vp, vp, vp, vp, vp, vp, ctypes.c_double, ctypes.c_double, vp],
        "fnpf_laplace_solve_vjp": [vp, vp, vp, vp, vp, vp, vp, vp, vp],
        "fnpf_tape_begin": [vp, ctypes.c_int],
        "fnpf_tape_end": [vp],
        "fnpf_step_adjoint_taped": [vp, ctypes.c_int, vp, vp, vp, vp, vp, ctypes.c_double, vp],
        "fnpf_ensemble_create": [ctypes.POINTER(vp), ctypes.c_int, ctypes.POINTER(vp)],
        "fnpf_ensemble_set_batching": [vp, ctypes.c_int, ctypes.c_int, ctypes.c_int64],
        "fnpf_ensemble_stats": [vp, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                                ctypes.POINTER(ctypes.c_int64)],
        "fnpf_prism_numbering": [vp, ctypes.c_int, vp, ctypes.c_int, ctypes.c_int, vp, vp, vp,
                                 ctypes.POINTER(ctypes.c_int)],
        "fnpf_prism_tables": [ctypes.c_int, vp, vp, vp, vp, ctypes.POINTER(ctypes.c_int)],
        "fnpf_prism_create": [vp, ctypes.c_int, vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.POINTER(vp)],
        "fnpf_prism_sizes": [vp, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int64)],
        "fnpf_prism_apply": [vp, vp, vp, vp, vp, vp],
        "fnpf_prism_diagonal": [vp, vp, vp, vp, vp],
        "fnpf_prism_set_filter": [vp, ctypes.POINTER(Filter)],
        "fnpf_prism_filter_apply": [vp, vp, vp],
        "fnpf_prism_apply_stored": [vp, vp, vp, vp, vp, vp],
        "fnpf_prism_laplace_solve": [vp, ctypes.POINTER(PrismOpts), vp, vp, vp, vp, ctypes.POINTER(SolveInfo), vp],
        "fnpf_prism_precond_apply": [vp, ctypes.POINTER(PrismOpts), vp, vp, vp, vp, vp],
        "fnpf_prism_laplace_solve_vjp": [vp, ctypes.POINTER(PrismOpts), vp, vp, vp, vp, vp, vp, vp,
                                         ctypes.POINTER(SolveInfo), vp],
        "fnpf_prism_step_adjoint": [vp, ctypes.POINTER(PrismOpts), vp, vp, vp, vp, vp, vp, vp, vp, ctypes.c_double,
                                    ctypes.c_double, vp],
        "fnpf_prism_dtn": [vp, ctypes.POINTER(PrismOpts), vp, vp, vp, vp, ctypes.POINTER(SolveInfo), vp],
        "fnpf_prism_rhs": [vp, ctypes.POINTER(PrismOpts), vp, vp, vp, vp, vp, ctypes.POINTER(SolveInfo), vp],
        "fnpf_prism_rk4_step": [vp, ctypes.POINTER(PrismOpts), vp, vp, vp, ctypes.c_double, ctypes.c_double,
                                ctypes.POINTER(SolveInfo), vp],
        "fnpf_prism_set_relaxation": [vp, ctypes.POINTER(Relaxation)],
        "fnpf_prism_invariants": [vp, ctypes.POINTER(PrismOpts), vp, vp, vp, ctypes.POINTER(ctypes.c_double),
                                  ctypes.POINTER(ctypes.c_double), ctypes.POINTER(SolveInfo), vp],
        "fnpf_ensemble_rk4_step": [vp, ctypes.POINTER(vp), ctypes.POINTER(vp), ctypes.POINTER(ctypes.c_double),
                                   ctypes.POINTER(ctypes.c_double), ctypes.POINTER(SolveInfo), vp],
        "fnpf_autotune": [vp, vp, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int), vp],
        "fnpf_set_shapes": [vp, ctypes.c_int, ctypes.c_int],
        "fnpf_get_shapes": [vp] + [ctypes.POINTER(ctypes.c_int)] * 4,
        "fnpf_profile_enable": [vp, ctypes.c_int],
        "fnpf_profile_read": [vp, ctypes.POINTER(ctypes.c_double), i64p, i64p, ctypes.c_int],
        "fnpf_profile_read_fp32": [vp, ctypes.POINTER(ctypes.c_double), i64p],
    }
    for name, args in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = ctypes.c_int
    lib.fnpf_destroy_mesh.argtypes = [vp]
    lib.fnpf_destroy_mesh.restype = None
    lib.fnpf_default_opts.argtypes = [ctypes.POINTER(Opts)]
    lib.fnpf_default_opts.restype = None
    lib.fnpf_last_error.argtypes = [vp]
    lib.fnpf_last_error.restype = ctypes.c_char_p
    lib.fnpf_ensemble_destroy.argtypes = [vp]
    lib.fnpf_ensemble_destroy.restype = None
    lib.fnpf_ensemble_last_error.argtypes = [vp]
    lib.fnpf_ensemble_last_error.restype = ctypes.c_char_p
    lib.fnpf_prism_destroy.argtypes = [vp]
    lib.fnpf_prism_destroy.restype = None
    lib.fnpf_prism_default_opts.argtypes = [ctypes.POINTER(PrismOpts)]
    lib.fnpf_prism_default_opts.restype = None
    lib.fnpf_prism_last_error.argtypes = [vp]
    lib.fnpf_prism_last_error.restype = ctypes.c_char_p
    lib.fnpf_status_string.argtypes = [ctypes.c_int]
    lib.fnpf_status_string.restype = ctypes.c_char_p
    return lib


_LIB = load()


class FnpfError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("fnpf status %d (%s): %s" % (status, _LIB.fnpf_status_string(status).decode(), msg))
        self.status = status


def lib():
    return _LIB


def default_opts(**kw):
    o = Opts()
    _LIB.fnpf_default_opts(ctypes.byref(o))
    for k, v in kw.items():
        setattr(o, k, v)
    return o


def _check_meta(t, n, dtype, name):
    import torch
    want = getattr(torch, dtype)
    if t.dtype != want:
        raise ValueError("%s: expected dtype %s, got %s" % (name, want, t.dtype))
    if n is not None and t.numel() != n:
        raise ValueError("%s: expected %d elements, got %d" % (name, n, t.numel()))


def _ptr(t, n=None, dtype="float64", device=None, name="tensor"):
    """Device pointer of a contiguous CUDA tensor (or None -> NULL).

    The C ABI receives bare pointers and trusts their lengths, so every array
    is checked here before a call: of the expected dtype, with exactly n
    elements (when n is given), a contiguous CUDA tensor on `device` (the
    mesh's device; default: the current device).  A mismatch raises
    ValueError before anything is enqueued."""
    if t is None:
        return None
    import torch
    _check_meta(t, n, dtype, name)
    if not t.is_cuda or not t.is_contiguous():
        raise ValueError("%s: expected a contiguous CUDA tensor" % name)
    dev = torch.cuda.current_device() if device is None else device
    if t.device.index != dev:
        raise ValueError("%s: on cuda:%d, expected cuda:%d" % (name, t.device.index, dev))
    return ctypes.c_void_p(t.data_ptr())


def _ptrs(device, *specs):
    """Checked pointers of several arrays, spec = (tensor, n, dtype, name):
    dtypes and lengths of all of them first, then placement, so that a wrong
    size is reported as such whatever the order of the arguments."""
    for t, n, dtype, name in specs:
        if t is not None:
            _check_meta(t, n, dtype, name)
    return [_ptr(t, n, dtype, device, name) for t, n, dtype, name in specs]


def _stream(stream):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def make_desc(dim, nx, ny, nz, p, periodic_x, periodic_y, h, Lx=1.0, Ly=1.0, X=None, Y=None, g=9.81):
    """Builds a MeshDesc; returns (desc, keepalive) -- the arrays must outlive the call."""
    h = np.ascontiguousarray(h, dtype=np.float64)
    keep = [h]
    d = MeshDesc(dim=dim, nx=nx, ny=ny, nz=nz, p=p, periodic_x=int(periodic_x), periodic_y=int(periodic_y),
                 horiz_kind=FNPF_BOX if X is None else FNPF_ISOPARAMETRIC, Lx=Lx, Ly=Ly, g=g)
    d.h = h.ctypes.data_as(_dp)
    if X is not None:
        X = np.ascontiguousarray(X, dtype=np.float64)
        Y = np.ascontiguousarray(Y if Y is not None else np.zeros_like(X), dtype=np.float64)
        keep += [X, Y]
        d.X = X.ctypes.data_as(_dp)
        d.Y = Y.ctypes.data_as(_dp)
    return d, keep


def count_dofs(dim, nx, ny, nz, p, periodic_x=True, periodic_y=True):
    d = MeshDesc(dim=dim, nx=nx, ny=ny, nz=nz, p=p, periodic_x=int(periodic_x), periodic_y=int(periodic_y),
                 horiz_kind=FNPF_BOX, Lx=1.0, Ly=1.0, g=9.81)
    nv, ns = ctypes.c_int64(), ctypes.c_int64()
    st = _LIB.fnpf_count_dofs(ctypes.byref(d), ctypes.byref(nv), ctypes.byref(ns))
    if st != FNPF_OK:
        raise FnpfError(st, "bad descriptor")
    return nv.value, ns.value


def apply_noalloc(dim, nx, ny, nz, p, periodic_x, periodic_y, Lx, Ly, h, eta, x, y, stream=None):
    """y = A(eta) x for a box mesh without any device allocation (fnpf_apply_noalloc);
    h, eta, x, y are CUDA tensors."""
    d = MeshDesc(dim=dim, nx=nx, ny=ny, nz=nz, p=p, periodic_x=int(periodic_x), periodic_y=int(periodic_y),
                 horiz_kind=FNPF_BOX, Lx=Lx, Ly=Ly, g=9.81)
    # the entry point gets no array lengths: derive them from the box here
    # (fnpf_count_dofs is host arithmetic) and check every tensor against them
    n, ns = count_dofs(dim, nx, ny, nz, p, periodic_x, periodic_y)
    f64 = "float64"
    args = _ptrs(None, (h, ns, f64, "h"), (eta, ns, f64, "eta"), (x, n, f64, "x"), (y, n, f64, "y"))
    st = _LIB.fnpf_apply_noalloc(ctypes.byref(d), *args, _stream(stream))
    if st != FNPF_OK:
        raise FnpfError(st, _LIB.fnpf_last_error(None).decode())


def fma_probe(precision, blocks, iters, out, stream=None):
    """Enqueues the FMA-throughput probe (fnpf_fma_probe) on `stream`;
    `out` is a one-element CUDA tensor of the probe's precision.  Returns the
    floating-point operations of the launch."""
    dtype = "float64" if precision == FNPF_FP64 else "float32"
    fl = ctypes.c_double()
    st = _LIB.fnpf_fma_probe(int(precision), int(blocks), int(iters), _ptr(out, 1, dtype, name="out"),
                             ctypes.byref(fl), _stream(stream))
    if st != FNPF_OK:
        raise FnpfError(st, "fma probe")
    return fl.value


class Mesh:
    """Owns one fnpf_mesh (device workspaces on the current CUDA device)."""

    def __init__(self, dim, nx, ny, nz, p, periodic_x=True, periodic_y=True, h=None, Lx=1.0, Ly=1.0, X=None,
                 Y=None, g=9.81, opts=None):
        if h is None:
            raise ValueError("h (depth at surface nodes) is required")
        d, keep = make_desc(dim, nx, ny, nz, p, periodic_x, periodic_y, h, Lx, Ly, X, Y, g)
        o = opts if opts is not None else default_opts()
        handle = ctypes.c_void_p()
        st = _LIB.fnpf_create_mesh(ctypes.byref(d), ctypes.byref(o), ctypes.byref(handle))
        if st != FNPF_OK:
            raise FnpfError(st, _LIB.fnpf_last_error(None).decode())
        self._h = handle
        self.g = g
        self._depth = np.array(keep[0], dtype=np.float64)   # host copy of the depth the mesh was created with
        self.dim, self.nx, self.ny, self.nz, self.p = dim, nx, (ny if dim == 3 else 1), nz, p
        self.periodic_x, self.periodic_y = bool(periodic_x), bool(periodic_y) and dim == 3
        nv, ns = ctypes.c_int64(), ctypes.c_int64()
        _LIB.fnpf_mesh_sizes(self._h, ctypes.byref(nv), ctypes.byref(ns))
        self.N, self.ns = nv.value, ns.value
        self.n_interior = self.N - self.ns
        import torch
        self.device = torch.cuda.current_device()   # the device the mesh's memory lives on

    def _args(self, *specs, dtype="float64"):
        """Checked pointers of this mesh's arrays, spec = (tensor, name, kind):
        kind "s" a surface field [Ns], "v" a volume field [N], "i" the
        interior unknowns [N_I]."""
        size = {"s": self.ns, "v": self.N, "i": self.n_interior}
        return _ptrs(self.device, *[(t, size[k], dtype, nm) for t, nm, k in specs])

    def close(self):
        if getattr(self, "_h", None):
            _LIB.fnpf_destroy_mesh(self._h)
            self._h = None

    def __del__(self):
        self.close()

    def _check(self, st):
        if st != FNPF_OK:
            raise FnpfError(st, _LIB.fnpf_last_error(self._h).decode())

    def depth(self):
        """The still-water depth h [Ns] the mesh was created with (a host
        float64 tensor)."""
        import torch
        return torch.from_numpy(self._depth.copy())

    def set_opts(self, opts):
        self._check(_LIB.fnpf_set_opts(self._h, ctypes.byref(opts)))

    def surface_coords(self):
        x = np.zeros(self.ns)
        y = np.zeros(self.ns)
        self._check(_LIB.fnpf_surface_coords(self._h, x.ctypes.data_as(_dp), y.ctypes.data_as(_dp)))
        return x, y

    def apply(self, eta, x, y, stream=None):
        a = self._args((eta, "eta", "s"), (x, "x", "v"), (y, "y", "v"))
        self._check(_LIB.fnpf_apply(self._h, *a, _stream(stream)))

    def apply_f32(self, eta, x, y, stream=None):
        a = self._args((eta, "eta", "s"), (x, "x", "v"), (y, "y", "v"), dtype="float32")
        self._check(_LIB.fnpf_apply_f32(self._h, *a, _stream(stream)))

    def diagonal(self, eta, d, stream=None):
        self._check(_LIB.fnpf_diagonal(self._h, *self._args((eta, "eta", "s"), (d, "d", "v")), _stream(stream)))

    def set_filter(self, alpha, order=2, cutoff=0):
        """Modal filter of eta and phi after every RK4 step (alpha = 0: off)."""
        f = Filter(float(alpha), int(order), int(cutoff))
        self._check(_LIB.fnpf_set_filter(self._h, ctypes.byref(f)))

    def set_dealias(self, points):
        """Over-integrated Zakharov right-hand sides on `points` Gauss points per
        direction (0: collocation)."""
        self._check(_LIB.fnpf_set_dealias(self._h, int(points)))

    def filter_apply(self, f, stream=None):
        self._check(_LIB.fnpf_filter_apply(self._h, *self._args((f, "f", "s")), _stream(stream)))

    def precond_apply(self, eta, r, z, stream=None):
        """z = M r, the FP64 preconditioner (p-multigrid V-cycle or Jacobi) set
        up from eta; r, z have the N_I interior unknowns."""
        a = self._args((eta, "eta", "s"), (r, "r", "i"), (z, "z", "i"))
        self._check(_LIB.fnpf_precond_apply(self._h, *a, _stream(stream)))

    def laplace_solve(self, eta, phis, phi, stream=None, info=True, check=True):
        inf = SolveInfo() if info else None
        a = self._args((eta, "eta", "s"), (phis, "phis", "s"), (phi, "phi", "v"))
        st = _LIB.fnpf_laplace_solve(self._h, *a,
                                     ctypes.byref(inf) if inf is not None else None, _stream(stream))
        if check:
            self._check(st)
        return inf.as_dict() if inf is not None else st

    def dtn(self, eta, phis, w, stream=None, info=True, check=True):
        inf = SolveInfo() if info else None
        a = self._args((eta, "eta", "s"), (phis, "phis", "s"), (w, "w", "s"))
        st = _LIB.fnpf_dtn(self._h, *a,
                           ctypes.byref(inf) if inf is not None else None, _stream(stream))
        if check:
            self._check(st)
        return inf.as_dict() if inf is not None else st

    def zakharov_rhs(self, eta, phis, w, deta, dphis, stream=None):
        a = self._args((eta, "eta", "s"), (phis, "phis", "s"), (w, "w", "s"), (deta, "deta", "s"),
                       (dphis, "dphis", "s"))
        self._check(_LIB.fnpf_zakharov_rhs(self._h, *a, _stream(stream)))

    def set_relaxation(self, cr, gen, amp=0.0, kx=0.0, ky=0.0, omega=1.0, phase=0.0, ramp_time=1.0):
        """Relaxation zones applied after every RK4 step (cr=None removes them)."""
        if cr is None:
            r = Relaxation(omega=1.0, ramp_time=1.0)
            self._check(_LIB.fnpf_set_relaxation(self._h, ctypes.byref(r)))
            return
        cr = np.ascontiguousarray(cr, dtype=np.float64)
        gen = np.ascontiguousarray(gen, dtype=np.float64)
        r = Relaxation(amp=amp, kx=kx, ky=ky, omega=omega, phase=phase, ramp_time=ramp_time)
        r.cr = cr.ctypes.data_as(_dp)
        r.gen = gen.ctypes.data_as(_dp)
        self._check(_LIB.fnpf_set_relaxation(self._h, ctypes.byref(r)))

    def step_adjoint(self, eta, phis, lam_eta, lam_phis, lam_eta_out, lam_phis_out, lam_h=None, t=0.0, dt=0.01,
                     stream=None):
        """dJ/dy_n from dJ/dy_{n+1} for one RK4 step from (eta, phis); adds dJ/dh into lam_h."""
        args = self._args(*[(t_, n_, "s") for t_, n_ in ((eta, "eta"), (phis, "phis"), (lam_eta, "lam_eta"),
                                                          (lam_phis, "lam_phis"), (lam_eta_out, "lam_eta_out"),
                                                          (lam_phis_out, "lam_phis_out"), (lam_h, "lam_h"))])
        self._check(_LIB.fnpf_step_adjoint(self._h, *args, float(t), float(dt), _stream(stream)))

    def invariants(self, eta, phis, stream=None):
        """(mass, energy) of the state: M = sum W eta, E = 1/2 phi^T A phi +
        1/2 g sum W eta^2 (fnpf_invariants; one Laplace solve)."""
        a = self._args((eta, "eta", "s"), (phis, "phis", "s"))
        ms, en = ctypes.c_double(), ctypes.c_double()
        self._check(_LIB.fnpf_invariants(self._h, *a, ctypes.byref(ms), ctypes.byref(en), None,
                                         _stream(stream)))
        return ms.value, en.value

    def laplace_solve_vjp(self, eta, phis, phi, gbar, lam_eta, lam_phis, lam_h=None, stream=None):
        """Adds the cotangents of (eta, phis[, h]) for a cotangent gbar [N] of
        the potential phi = laplace_solve(eta, phis) (fnpf_laplace_solve_vjp)."""
        a = self._args((eta, "eta", "s"), (phis, "phis", "s"), (phi, "phi", "v"), (gbar, "gbar", "v"),
                       (lam_eta, "lam_eta", "s"), (lam_phis, "lam_phis", "s"), (lam_h, "lam_h", "s"))
        self._check(_LIB.fnpf_laplace_solve_vjp(self._h, *a, _stream(stream)))

    def tape_begin(self, capacity):
        """Record the stage data of the next `capacity` RK4 steps (slots 0, 1, ...)."""
        self._check(_LIB.fnpf_tape_begin(self._h, int(capacity)))

    def tape_end(self):
        self._check(_LIB.fnpf_tape_end(self._h))

    def step_adjoint_taped(self, slot, lam_eta, lam_phis, lam_eta_out, lam_phis_out, lam_h=None, dt=0.01,
                           stream=None):
        """fnpf_step_adjoint for the step recorded in tape slot `slot` (no forward recompute)."""
        args = self._args(*[(t_, n_, "s") for t_, n_ in ((lam_eta, "lam_eta"), (lam_phis, "lam_phis"),
                                                          (lam_eta_out, "lam_eta_out"),
                                                          (lam_phis_out, "lam_phis_out"), (lam_h, "lam_h"))])
        self._check(_LIB.fnpf_step_adjoint_taped(self._h, int(slot), *args, float(dt), _stream(stream)))

    def set_shapes(self, variant64, variant32):
        self._check(_LIB.fnpf_set_shapes(self._h, int(variant64), int(variant32)))

    def get_shapes(self):
        """(variant64, variant32, columns per CTA fp64, columns per CTA fp32)."""
        v = [ctypes.c_int() for _ in range(4)]
        self._check(_LIB.fnpf_get_shapes(self._h, *[ctypes.byref(x) for x in v]))
        return tuple(x.value for x in v)

    def autotune(self, eta, stream=None):
        v64, v32 = ctypes.c_int(), ctypes.c_int()
        a = self._args((eta, "eta", "s"))
        self._check(_LIB.fnpf_autotune(self._h, *a, ctypes.byref(v64), ctypes.byref(v32), _stream(stream)))
        return v64.value, v32.value

    def profile_enable(self, on=True):
        self._check(_LIB.fnpf_profile_enable(self._h, int(on)))

    def profile_read(self, reset=False):
        ms, cnt, launches = ctypes.c_double(), ctypes.c_int64(), ctypes.c_int64()
        ms32, cnt32 = ctypes.c_double(), ctypes.c_int64()
        self._check(_LIB.fnpf_profile_read_fp32(self._h, ctypes.byref(ms32), ctypes.byref(cnt32)))
        self._check(_LIB.fnpf_profile_read(self._h, ctypes.byref(ms), ctypes.byref(cnt), ctypes.byref(launches),
                                           int(reset)))
        return dict(apply_ms=ms.value, apply_count=cnt.value, launches=launches.value, apply32_ms=ms32.value,
                    apply32_count=cnt32.value)

    def rk4_step(self, eta, phis, t, dt, stream=None, info=False, check=True):
        infos = (SolveInfo * 4)() if info else None
        a = self._args((eta, "eta", "s"), (phis, "phis", "s"))
        st = _LIB.fnpf_rk4_step(self._h, *a, float(t), float(dt), infos, _stream(stream))
        if check:
            self._check(st)
        return [i.as_dict() for i in infos] if infos is not None else st


class Ensemble:
    """Independent tanks advanced together, one CUDA graph launch per RK4 step
    (fnpf_ensemble_*).  The meshes must stay alive while the ensemble exists."""

    def __init__(self, meshes):
        self.meshes = list(meshes)
        arr = (ctypes.c_void_p * len(self.meshes))(*[m._h.value for m in self.meshes])
        h = ctypes.c_void_p()
        st = _LIB.fnpf_ensemble_create(arr, len(self.meshes), ctypes.byref(h))
        if st != FNPF_OK:
            raise FnpfError(st, _LIB.fnpf_ensemble_last_error(None).decode())
        self._h = h

    def close(self):
        if getattr(self, "_h", None):
            _LIB.fnpf_ensemble_destroy(self._h)
            self._h = None

    def __del__(self):
        self.close()

    def set_batching(self, on, max_tanks=0, max_dof=0):
        """Batched groups (True, the default) or one branch of per-tank kernels
        per tank (False), groups of at most max_tanks tanks (0: 32) and max_dof
        degrees of freedom (0: no limit), from the next step on."""
        st = _LIB.fnpf_ensemble_set_batching(self._h, 1 if on else 0, int(max_tanks), int(max_dof))
        if st != FNPF_OK:
            raise FnpfError(st, _LIB.fnpf_ensemble_last_error(self._h).decode())

    def stats(self):
        """{"groups", "batched_tanks", "kernels"}: batched groups and their tanks
        in the current graph, kernels launched by the last ensemble step."""
        g, b, k = ctypes.c_int(), ctypes.c_int(), ctypes.c_int64()
        st = _LIB.fnpf_ensemble_stats(self._h, ctypes.byref(g), ctypes.byref(b), ctypes.byref(k))
        if st != FNPF_OK:
            raise FnpfError(st, _LIB.fnpf_ensemble_last_error(self._h).decode())
        return {"groups": g.value, "batched_tanks": b.value, "kernels": k.value}

    def rk4_step(self, etas, phiss, ts, dts, stream=None, info=False):
        n = len(self.meshes)
        if len(etas) != n or len(phiss) != n or len(ts) != n or len(dts) != n:
            raise ValueError("expected one state, time and step size per tank (%d)" % n)
        ptrs = [m._args((a, "etas[%d]" % i, "s"), (b, "phiss[%d]" % i, "s"))
                for i, (m, a, b) in enumerate(zip(self.meshes, etas, phiss))]
        e = (ctypes.c_void_p * n)(*[q[0].value for q in ptrs])
        p = (ctypes.c_void_p * n)(*[q[1].value for q in ptrs])
        tt = (ctypes.c_double * n)(*[float(v) for v in ts])
        dd = (ctypes.c_double * n)(*[float(v) for v in dts])
        infos = (SolveInfo * (4 * n))() if info else None
        st = _LIB.fnpf_ensemble_rk4_step(self._h, e, p, tt, dd, infos, _stream(stream))
        if st != FNPF_OK:
            raise FnpfError(st, _LIB.fnpf_ensemble_last_error(self._h).decode())
        return [i.as_dict() for i in infos] if infos is not None else None


def _host_mesh_arrays(verts, tris):
    import numpy as np
    v = np.ascontiguousarray(verts, dtype=np.float64)
    t = np.ascontiguousarray(tris, dtype=np.int32)
    if v.ndim != 2 or v.shape[1] != 2 or t.ndim != 2 or t.shape[1] != 3:
        raise ValueError("verts must be [nverts, 2] and tris [ntris, 3]")
    return v, t


def prism_numbering(verts, tris, p):
    """(tnodes [ntris, (p+1)(p+2)/2], x [Ns], y [Ns]) of the order-p nodes of a
    triangle mesh (fnpf_prism_numbering; host only)."""
    import numpy as np
    v, t = _host_mesh_arrays(verts, tris)
    ns = ctypes.c_int()
    st = _LIB.fnpf_prism_numbering(v.ctypes.data, len(v), t.ctypes.data, len(t), int(p), None, None, None,
                                   ctypes.byref(ns))
    if st != FNPF_OK:
        raise FnpfError(st, "prism numbering")
    nt = (p + 1) * (p + 2) // 2
    tn = np.zeros((len(t), nt), dtype=np.int32)
    x, y = np.zeros(ns.value), np.zeros(ns.value)
    st = _LIB.fnpf_prism_numbering(v.ctypes.data, len(v), t.ctypes.data, len(t), int(p), tn.ctypes.data,
                                   x.ctypes.data, y.ctypes.data, ctypes.byref(ns))
    if st != FNPF_OK:
        raise FnpfError(st, "prism numbering")
    return tn, x, y


def prism_tables(p):
    """(L, Lr, Ls [nq, nt], wq [nq]): the nodal triangle basis and its r, s
    derivatives at the quadrature points (fnpf_prism_tables; host only)."""
    import numpy as np
    nq = ctypes.c_int()
    st = _LIB.fnpf_prism_tables(int(p), None, None, None, None, ctypes.byref(nq))
    if st != FNPF_OK:
        raise FnpfError(st, "prism tables")
    nt = (p + 1) * (p + 2) // 2
    L, Lr, Ls = (np.zeros((nq.value, nt)) for _ in range(3))
    wq = np.zeros(nq.value)
    st = _LIB.fnpf_prism_tables(int(p), L.ctypes.data, Lr.ctypes.data, Ls.ctypes.data, wq.ctypes.data,
                                ctypes.byref(nq))
    if st != FNPF_OK:
        raise FnpfError(st, "prism tables")
    return L, Lr, Ls, wq


class PrismMesh:
    """N_z layers of order-p prisms over an unstructured triangle mesh
    (fnpf_prism_*): y = A(eta, h) x on the device."""

    def __init__(self, verts, tris, p, nz):
        v, t = _host_mesh_arrays(verts, tris)
        h = ctypes.c_void_p()
        st = _LIB.fnpf_prism_create(v.ctypes.data, len(v), t.ctypes.data, len(t), int(p), int(nz), ctypes.byref(h))
        if st != FNPF_OK:
            raise FnpfError(st, _LIB.fnpf_prism_last_error(None).decode())
        self._h = h
        self.p, self.nz = int(p), int(nz)
        nv, ns = ctypes.c_int64(), ctypes.c_int64()
        _LIB.fnpf_prism_sizes(h, ctypes.byref(nv), ctypes.byref(ns))
        self.N, self.ns = nv.value, ns.value

    def close(self):
        if getattr(self, "_h", None):
            _LIB.fnpf_prism_destroy(self._h)
            self._h = None

    def __del__(self):
        self.close()

    def apply(self, eta, h, x, y, stream=None):
        ptrs = _ptrs(None, (eta, self.ns, "float64", "eta"), (h, self.ns, "float64", "h"),
                     (x, self.N, "float64", "x"), (y, self.N, "float64", "y"))
        st = _LIB.fnpf_prism_apply(self._h, *ptrs, _stream(stream))
        if st != FNPF_OK:
            raise FnpfError(st, _LIB.fnpf_prism_last_error(self._h).decode())

    @staticmethod
    def default_opts(**kw):
        """fnpf_prism_opts with the library's defaults, fields overridden by kw."""
        o = PrismOpts()
        _LIB.fnpf_prism_default_opts(ctypes.byref(o))
        for k, v in kw.items():
            setattr(o, k, v)
        return o

    def _check(self, st, infos=None):
        if st != FNPF_OK:
            raise FnpfError(st, _LIB.fnpf_prism_last_error(self._h).decode())
        return infos

    def diagonal(self, eta, h, diag, stream=None):
        ptrs = _ptrs(None, (eta, self.ns, "float64", "eta"), (h, self.ns, "float64", "h"),
                     (diag, self.N, "float64", "diag"))
        self._check(_LIB.fnpf_prism_diagonal(self._h, *ptrs, _stream(stream)))

    def apply_stored(self, eta, h, x, y, stream=None):
        ptrs = _ptrs(None, (eta, self.ns, "float64", "eta"), (h, self.ns, "float64", "h"),
                     (x, self.N, "float64", "x"), (y, self.N, "float64", "y"))
        self._check(_LIB.fnpf_prism_apply_stored(self._h, *ptrs, _stream(stream)))

    def precond_apply(self, eta, h, r, z, opts=None, stream=None):
        """z [N] = the preconditioner of opts (Jacobi or one V-cycle) applied to
        the interior entries of r [N]."""
        ptrs = _ptrs(None, (eta, self.ns, "float64", "eta"), (h, self.ns, "float64", "h"),
                     (r, self.N, "float64", "r"), (z, self.N, "float64", "z"))
        st = _LIB.fnpf_prism_precond_apply(self._h, None if opts is None else ctypes.byref(opts), *ptrs,
                                           _stream(stream))
        self._check(st)

    def laplace_solve(self, eta, h, phis, phi, opts=None, stream=None):
        """phi [N] (in: interior guess) = the potential with phi = phis on the
        surface; returns the solve's info as a dict."""
        ptrs = _ptrs(None, (eta, self.ns, "float64", "eta"), (h, self.ns, "float64", "h"),
                     (phis, self.ns, "float64", "phis"), (phi, self.N, "float64", "phi"))
        info = SolveInfo()
        st = _LIB.fnpf_prism_laplace_solve(self._h, None if opts is None else ctypes.byref(opts), *ptrs,
                                           ctypes.byref(info), _stream(stream))
        return self._check(st, info.as_dict())

    def laplace_solve_vjp(self, eta, h, phi, lam_phi, lam_eta, lam_phis, lam_h=None, opts=None, stream=None):
        """dJ/deta, dJ/dphis (and dJ/dh) [Ns] of the solve phi [N] for the
        cotangent lam_phi = dJ/dphi [N]; returns the adjoint solve's info."""
        ptrs = _ptrs(None, (eta, self.ns, "float64", "eta"), (h, self.ns, "float64", "h"),
                     (phi, self.N, "float64", "phi"), (lam_phi, self.N, "float64", "lam_phi"),
                     (lam_eta, self.ns, "float64", "lam_eta"), (lam_phis, self.ns, "float64", "lam_phis"),
                     (lam_h, self.ns, "float64", "lam_h"))
        info = SolveInfo()
        st = _LIB.fnpf_prism_laplace_solve_vjp(self._h, None if opts is None else ctypes.byref(opts), *ptrs,
                                               ctypes.byref(info), _stream(stream))
        return self._check(st, info.as_dict())

    def step_adjoint(self, h, eta_n, phis_n, lam_eta, lam_phis, lam_eta_out, lam_phis_out, dt, lam_h=None,
                     opts=None, stream=None, t=0.0):
        """dJ/d(eta, phis)_n (and dJ/dh) of one RK4 step from (eta_n, phis_n) for
        the cotangents (lam_eta, lam_phis) of its result [Ns each]."""
        ptrs = _ptrs(None, (h, self.ns, "float64", "h"), (eta_n, self.ns, "float64", "eta_n"),
                     (phis_n, self.ns, "float64", "phis_n"), (lam_eta, self.ns, "float64", "lam_eta"),
                     (lam_phis, self.ns, "float64", "lam_phis"), (lam_eta_out, self.ns, "float64", "lam_eta_out"),
                     (lam_phis_out, self.ns, "float64", "lam_phis_out"), (lam_h, self.ns, "float64", "lam_h"))
        st = _LIB.fnpf_prism_step_adjoint(self._h, None if opts is None else ctypes.byref(opts), *ptrs, float(t),
                                          float(dt), _stream(stream))
        self._check(st)

    def dtn(self, eta, h, phis, w, opts=None, stream=None):
        ptrs = _ptrs(None, (eta, self.ns, "float64", "eta"), (h, self.ns, "float64", "h"),
                     (phis, self.ns, "float64", "phis"), (w, self.ns, "float64", "w"))
        info = SolveInfo()
        st = _LIB.fnpf_prism_dtn(self._h, None if opts is None else ctypes.byref(opts), *ptrs, ctypes.byref(info),
                                 _stream(stream))
        return self._check(st, info.as_dict())

    def rhs(self, eta, h, phis, k_eta, k_phis, opts=None, stream=None):
        ptrs = _ptrs(None, (eta, self.ns, "float64", "eta"), (h, self.ns, "float64", "h"),
                     (phis, self.ns, "float64", "phis"), (k_eta, self.ns, "float64", "k_eta"),
                     (k_phis, self.ns, "float64", "k_phis"))
        info = SolveInfo()
        st = _LIB.fnpf_prism_rhs(self._h, None if opts is None else ctypes.byref(opts), *ptrs, ctypes.byref(info),
                                 _stream(stream))
        return self._check(st, info.as_dict())

    def set_filter(self, alpha, order=2, cutoff=0):
        """The modal filter of the triangular surface elements (alpha = 0: off);
        every later rk4_step filters eta and phis."""
        f = Filter(float(alpha), int(order), int(cutoff))
        self._check(_LIB.fnpf_prism_set_filter(self._h, ctypes.byref(f)))

    def filter_apply(self, f, stream=None):
        ptrs = _ptrs(None, (f, self.ns, "float64", "f"))
        self._check(_LIB.fnpf_prism_filter_apply(self._h, *ptrs, _stream(stream)))

    def invariants(self, eta, h, phis, opts=None, stream=None):
        """(mass, energy) of the state (eta, phis) [Ns] (waits for the stream)."""
        ptrs = _ptrs(None, (eta, self.ns, "float64", "eta"), (h, self.ns, "float64", "h"),
                     (phis, self.ns, "float64", "phis"))
        M, En, info = ctypes.c_double(), ctypes.c_double(), SolveInfo()
        st = _LIB.fnpf_prism_invariants(self._h, None if opts is None else ctypes.byref(opts), *ptrs,
                                        ctypes.byref(M), ctypes.byref(En), ctypes.byref(info), _stream(stream))
        self._check(st)
        return M.value, En.value

    def set_relaxation(self, cr, gen, amp, kx, ky, omega, phase, ramp_time):
        """Relaxation zones (host arrays cr, gen [Ns]); cr None removes them."""
        if cr is None:
            self._check(_LIB.fnpf_prism_set_relaxation(self._h, None))
            return
        c = np.ascontiguousarray(cr, dtype=np.float64)
        g = np.ascontiguousarray(gen, dtype=np.float64)
        if c.shape != (self.ns,) or g.shape != (self.ns,):
            raise ValueError("cr and gen must have Ns = %d entries" % self.ns)
        r = Relaxation(c.ctypes.data_as(_dp), g.ctypes.data_as(_dp), amp, kx, ky, omega, phase, ramp_time)
        self._check(_LIB.fnpf_prism_set_relaxation(self._h, ctypes.byref(r)))

    def rk4_step(self, h, eta, phis, dt, opts=None, stream=None, t=0.0):
        """One RK4 step of (eta, phis) from t to t + dt in place (then the
        relaxation zones and the modal filter, when set); returns the four
        stages' infos."""
        ptrs = _ptrs(None, (h, self.ns, "float64", "h"), (eta, self.ns, "float64", "eta"),
                     (phis, self.ns, "float64", "phis"))
        infos = (SolveInfo * 4)()
        st = _LIB.fnpf_prism_rk4_step(self._h, None if opts is None else ctypes.byref(opts), *ptrs, float(t),
                                      float(dt), infos, _stream(stream))
        return self._check(st, [infos[i].as_dict() for i in range(4)])
