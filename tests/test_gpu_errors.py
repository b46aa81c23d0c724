"""Failure detection through status codes (no GPU fault is provoked: every
failure is made on the host side -- bad descriptors, non-finite or folded
inputs, an iteration cap)."""
import math

import numpy as np
import pytest
import torch

from tests.pairs import Case

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("bad", [dict(p=0), dict(p=9), dict(nx=0), dict(nx=1), dict(nz=0)])
def test_create_rejects_bad_descriptor(fnpf, bad):
    args = dict(dim=3, nx=3, ny=2, nz=1, p=3)
    args.update(bad)
    ncx = max(1, args["p"] * max(args["nx"], 1))
    h = np.full(ncx * max(1, args["p"] * 2), 0.5)
    with pytest.raises(fnpf.FnpfError) as e:
        fnpf.Mesh(args["dim"], args["nx"], args["ny"], args["nz"], args["p"], True, True, h)
    assert e.value.status == fnpf.FNPF_EINVAL


def test_create_rejects_nonpositive_depth(fnpf):
    h = np.full(6 * 4, 0.5)
    h[5] = 0.0
    with pytest.raises(fnpf.FnpfError) as e:
        fnpf.Mesh(3, 3, 2, 1, 2, True, True, h)
    assert e.value.status == fnpf.FNPF_EINVAL


def test_nan_input_reports_diverged(fnpf):
    c = Case(fnpf, 3, 3, 2, 2, 3, True, True)
    eta = c.eta.copy()
    eta[3] = math.nan
    phi = torch.zeros(c.om.N, dtype=torch.float64, device=c.dev)
    info = c.gm.laplace_solve(c.t(eta), c.t(c.phis), phi, check=False)
    assert info["status"] == fnpf.FNPF_EDIVERGED


def test_folded_mesh_reports_diverged(fnpf):
    c = Case(fnpf, 3, 3, 2, 2, 3, True, True)
    eta = c.eta.copy()
    eta[7] = -2 * c.h[7]
    w = torch.zeros(c.om.ns, dtype=torch.float64, device=c.dev)
    with pytest.raises(fnpf.FnpfError) as e:
        c.gm.dtn(c.t(eta), c.t(c.phis), w)
    assert e.value.status == fnpf.FNPF_EDIVERGED


def test_iteration_cap_reports_noconv_and_mesh_stays_usable(fnpf):
    c = Case(fnpf, 3, 4, 3, 2, 4, True, True, opts=fnpf.default_opts(max_iter=2, rtol=1e-12))
    phi = torch.zeros(c.om.N, dtype=torch.float64, device=c.dev)
    info = c.gm.laplace_solve(c.t(c.eta), c.t(c.phis), phi, check=False)
    assert info["status"] == fnpf.FNPF_ENOCONV and info["iters"] == 2
    c.gm.set_opts(fnpf.default_opts(rtol=1e-12))
    info = c.gm.laplace_solve(c.t(c.eta), c.t(c.phis), phi)
    assert info["status"] == 0 and info["rel_res"] <= 1e-12
