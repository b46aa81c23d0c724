"""fnpf_apply_noalloc, the operator application for callers that cannot
allocate device memory (a plug-in inside an application that owns all device
memory through its own pool, or a loop with a fixed memory budget): called
through the C ABI, it must give the same y = A(eta) x as fnpf_apply, on two
calls in a row and a third in 2D (different meshes, so stale contents of the shared device
array from the first call would show up in the second).  Collected last on
purpose."""
import numpy as np
import pytest
import torch

from tests.pairs import Case, rel_max

pytestmark = pytest.mark.gpu


def test_noalloc_apply_matches_apply_on_two_calls(fnpf):
    shapes = [(3, 5, 4, 2, 5, True, False), (3, 3, 3, 3, 4, False, True), (2, 8, 1, 2, 4, True, False)]
    for k, shape in enumerate(shapes):
        c = Case(fnpf, *shape, seed=k)
        dim, nx, ny, nz, p, px, py = shape
        x = c.t(c.rng.standard_normal(c.om.N))
        eta, h = c.t(c.eta), c.t(c.h)
        y_ref = torch.empty_like(x)
        c.gm.apply(eta, x, y_ref)
        y = torch.full_like(x, float("nan"))
        fnpf.apply_noalloc(dim, nx, ny, nz, p, px, py, 1.0, 1.0, h, eta, x, y)
        torch.cuda.synchronize()
        assert rel_max(y.cpu().numpy(), y_ref.cpu().numpy()) < 1e-12


def test_noalloc_rejects_mesh_beyond_the_fixed_scratch(fnpf):
    """Called through the C ABI directly (the Python wrapper would reject the
    short arrays first): the library refuses a mesh whose tables and scratch
    exceed the fixed device array before it touches any array."""
    import ctypes
    dev = torch.device("cuda:0")
    t = torch.zeros(8, dtype=torch.float64, device=dev)
    d = fnpf.MeshDesc(dim=3, nx=200, ny=200, nz=4, p=6, periodic_x=1, periodic_y=1, horiz_kind=fnpf.FNPF_BOX,
                      Lx=1.0, Ly=1.0, g=9.81)
    ptr = ctypes.c_void_p(t.data_ptr())
    st = fnpf.lib().fnpf_apply_noalloc(ctypes.byref(d), ptr, ptr, ptr, ptr,
                                       ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == fnpf.FNPF_EINVAL
    assert "16 MiB" in fnpf.lib().fnpf_last_error(None).decode()
