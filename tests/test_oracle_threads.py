"""The oracle's per-ghost and per-cell loops run on several host threads
(OpenMP) for the timed CPU baseline; every ghost and every cell is computed
independently and the reductions stay serial, so the state, residual, forces
and ghost band are bitwise the same for any thread count."""
import os

import numpy as np
import pytest

import oracle
from paper_2512_20252_gb300 import workloads as wl


@pytest.mark.parametrize("make", [
    lambda: wl.small_2d("naca", n=40, nv=12, Ma=0.6),
    lambda: dict(wl.small_2d("ellipse", n=24, nv=10, Kn=0.08, Ma=0.5), upwind=3),
    lambda: wl._case(3, 12, 2.0, 8, 4.5, 0.1, 0.5, wl.sphere(0.6)),
])
def test_threads_give_bitwise_identical_results(make):
    case = make()
    nth = max(2, len(os.sched_getaffinity(0)))
    one = oracle.OracleCase(case, threads=1)
    many = oracle.OracleCase(case, threads=nth)
    assert many.threads == nth
    r1, rn = one.step(4), many.step(4)
    assert r1 == rn
    np.testing.assert_array_equal(one.get_f(), many.get_f())
    for a, b in zip(one.forces(), many.forces()):
        np.testing.assert_array_equal(a, b)
    g1, gn = one.ghost_band(), many.ghost_band()
    for k in g1:
        np.testing.assert_array_equal(g1[k], gn[k])
