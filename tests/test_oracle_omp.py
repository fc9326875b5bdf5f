"""The all-cores build of the oracle (the same C source compiled with OpenMP over its point
loops, used only to time the CPU baseline) gives the single-thread oracle's results bit for
bit: every point's arithmetic is unchanged and there are no reductions."""
import numpy as np

from paper_2504_03074_gb300 import grids as G
from paper_2504_03074_gb300 import grids3 as G3


def test_openmp_oracle_equals_single_thread_2d():
    from oracle import oracle as O
    prob = G.disk_problem(nb=128, nth=256, nr=16, order=4, omega=10.0, seed=3)
    v = G.random_state(prob, 4)
    a = O.Oracle(prob).iterate(v, True)
    b = O.Oracle(prob, openmp=True).iterate(v, True)
    assert np.array_equal(a, b)


def test_openmp_oracle_equals_single_thread_3d():
    from oracle import oracle3 as O3
    prob = G3.box_in_box_problem()
    v = G3.random_state3(prob, 5)
    assert np.array_equal(O3.Oracle3(prob).iterate(v, False),
                          O3.Oracle3(prob, openmp=True).iterate(v, False))
