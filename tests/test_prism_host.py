"""Host-side parts of the library's prism elements (no GPU): the order-p
surface numbering and the basis tables at the triangle quadrature points,
written in C++ independently of the oracle, against oracle/prism.py."""
import numpy as np
import pytest

from oracle import prism as P
from paper_2506_09435_gb300 import workloads as W


@pytest.fixture(scope="module")
def fnpf():
    from paper_2506_09435_gb300 import fnpf as f
    return f


@pytest.mark.parametrize("p", [1, 2, 3, 4, 6])
def test_numbering_matches_oracle(fnpf, p):
    v, t = W.triangulated_box(4, 3, 2.0, 1.0)
    tn, x, y = fnpf.prism_numbering(v, t, p)
    tm = P.TriMesh(v, t, p)
    assert tm.ns == len(x)
    assert np.array_equal(tn, tm.nodes)
    assert np.max(np.abs(x - tm.xs)) < 1e-14 and np.max(np.abs(y - tm.ys)) < 1e-14


@pytest.mark.parametrize("p", [1, 2, 3, 4, 5, 6, 7, 8])
def test_tables_match_oracle(fnpf, p):
    L, Lr, Ls, wq = fnpf.prism_tables(p)
    rq, sq, wo = P.tri_quadrature(p + 2)
    Lo, Lro, Lso = P.tri_basis(p, rq, sq)
    assert np.max(np.abs(wq - wo)) < 1e-15
    scale = max(1.0, np.max(np.abs(Lro)))
    for a, b in ((L, Lo), (Lr, Lro), (Ls, Lso)):
        assert np.max(np.abs(a - b)) < 1e-11 * scale, p


def test_bad_meshes_rejected(fnpf):
    v, t = W.triangulated_box(2, 2)
    for bad in (np.array([[0, 1, 99]]), np.array([[0, 0, 1]]), np.array([[-1, 1, 2]])):
        with pytest.raises(fnpf.FnpfError):
            fnpf.prism_numbering(v, bad, 2)
    with pytest.raises(ValueError):
        fnpf.prism_numbering(v[:, :1], t, 2)
