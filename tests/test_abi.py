"""The C ABI library loads and exports every entry point declared in
include/fnpf.h; host-only calls work without a GPU."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "fnpf.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(fnpf_[a-z0-9_]+)\s*\(", src)))


def test_exports_every_declared_symbol(fnpf):
    names = declared_functions()
    assert "fnpf_rk4_step" in names and "fnpf_create_mesh" in names
    lib = ctypes.CDLL(fnpf.LIB_PATH)
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_count_dofs_matches_paper_tables(fnpf):
    from tests.test_oracle_operator import read_dof_table
    for nx, ny, nz, p, nvol, nsurf, _ in read_dof_table():
        nv, ns = fnpf.count_dofs(3, nx, ny, nz, p, True, True)
        assert nv == nvol
        if nsurf >= 0:
            assert ns == nsurf


def test_count_dofs_walled_and_2d(fnpf):
    assert fnpf.count_dofs(3, 3, 2, 2, 4, False, False) == ((4 * 2 + 1) * 13 * 9, 13 * 9)
    assert fnpf.count_dofs(2, 8, 1, 2, 4, True, False) == (9 * 32, 32)


@pytest.mark.parametrize("bad", [dict(p=0), dict(p=9), dict(nx=0), dict(nz=0), dict(dim=4)])
def test_count_dofs_rejects_bad_descriptors(fnpf, bad):
    args = dict(dim=3, nx=2, ny=2, nz=1, p=3)
    args.update(bad)
    with pytest.raises(fnpf.FnpfError) as e:
        fnpf.count_dofs(args["dim"], args["nx"], args["ny"], args["nz"], args["p"])
    assert e.value.status == fnpf.FNPF_EINVAL


def test_default_opts(fnpf):
    o = fnpf.default_opts()
    assert o.precision == fnpf.FNPF_FP64 and o.rtol == 1e-10 and o.max_iter > 0 and o.check_every > 0
    assert o.coarse_iters == 6 and o.store_metric == 1 and o.coarse_solver == fnpf.FNPF_COARSE_CLUSTER
    assert o.cheb_kind == fnpf.FNPF_CHEB_FIRST and o.cheb_range == 160.0


def test_noalloc_wrapper_rejects_bad_tensors_before_any_call(fnpf):
    """fnpf_apply_noalloc gets no array lengths, so the binding checks dtype,
    length and placement first: a float32, a short or a host tensor raises
    ValueError before the library is called."""
    import torch
    n, ns = fnpf.count_dofs(3, 3, 2, 2, 4, True, False)
    good_s = torch.zeros(ns, dtype=torch.float64)
    good_v = torch.zeros(n, dtype=torch.float64)
    cases = [
        (good_s.float(), good_s, good_v, good_v, "dtype"),
        (good_s, good_s[:-1], good_v, good_v, "elements"),
        (good_s, good_s, good_v, torch.zeros(n - 7, dtype=torch.float64), "elements"),
        (good_s, good_s, good_v.float(), good_v, "dtype"),
        (good_s, good_s, good_v, good_v, "CUDA"),   # right sizes, but host memory
    ]
    for h, eta, x, y, what in cases:
        with pytest.raises(ValueError) as e:
            fnpf.apply_noalloc(3, 3, 2, 2, 4, True, False, 1.0, 1.0, h, eta, x, y)
        assert what in str(e.value)


def test_mesh_methods_check_lengths_and_dtypes(fnpf):
    """The Mesh methods check every tensor against the mesh's N and Ns (a
    stand-in object with those sizes, so no GPU is needed)."""
    import torch
    m = fnpf.Mesh.__new__(fnpf.Mesh)
    m._h, m.N, m.ns, m.n_interior, m.device = None, 90, 10, 80, 0
    eta = torch.zeros(10, dtype=torch.float64)
    with pytest.raises(ValueError, match="elements"):
        m.apply(eta, torch.zeros(89, dtype=torch.float64), torch.zeros(90, dtype=torch.float64))
    with pytest.raises(ValueError, match="dtype"):
        m.apply_f32(eta, torch.zeros(90, dtype=torch.float32), torch.zeros(90, dtype=torch.float32))
    with pytest.raises(ValueError, match="elements"):
        m.rk4_step(eta, torch.zeros(11, dtype=torch.float64), 0.0, 0.1)
    with pytest.raises(ValueError, match="elements"):
        m.precond_apply(eta, torch.zeros(90, dtype=torch.float64), torch.zeros(80, dtype=torch.float64))
    with pytest.raises(ValueError, match="dtype"):
        m.step_adjoint(eta, eta, eta, eta, eta, eta, torch.zeros(10, dtype=torch.float32))
