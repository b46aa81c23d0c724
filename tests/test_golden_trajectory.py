"""The stored oracle trajectory of the p = 6 tank (written by
tests/golden/make_box_p6_trajectory.py, which calls only the oracle) is what
the oracle computes now: its initial state is the seeded generator's, and one
oracle RK4 step from it reproduces the stored first step."""
import numpy as np

from oracle import surface
from tests.golden.make_box_p6_trajectory import OUT, initial_state


def test_stored_trajectory_is_the_oracles():
    ref = np.load(OUT)
    d, m, h, eta, phis, dt = initial_state()
    assert np.array_equal(ref["eta0"], eta) and np.array_equal(ref["phis0"], phis)
    assert np.array_equal(ref["h"], h) and float(ref["dt"]) == dt
    e1, p1 = surface.rk4_step(m, h, eta, phis, dt, d["g"], method="pcg")
    assert np.max(np.abs(e1 - ref["eta1"])) <= 1e-13 * np.max(np.abs(ref["eta1"]))
    assert np.max(np.abs(p1 - ref["phis1"])) <= 1e-13 * np.max(np.abs(ref["phis1"]))
    # the stored 20-step state is a genuine evolution of the wave, not a copy of the start
    assert np.linalg.norm(ref["eta20"] - eta) > 1e-2 * np.linalg.norm(eta)
