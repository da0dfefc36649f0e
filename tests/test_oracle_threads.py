"""The oracle's OpenMP loops give bit-identical results for every thread
count: each node's arithmetic is the same and no sum runs across nodes."""
import numpy as np

from oracle import oracle as o
from tests.cases import smooth_field


def _run(threads, nsteps=40):
    o.set_threads(threads)
    nx, ny = 37, 23
    L = o.Lattice(nx, ny, 1.0, 5.0, 1.9)
    L.set_law(o.NH, [1.5, 0.75])
    L.set_body_force(1e-3, -2e-3)
    L.set_edge(o.LEFT, o.VELOCITY)
    L.set_edge(o.RIGHT, o.TRACTION, (0.02, 0.01), o.T_SIN2_RAMP, (2.0, 0, 0, 0))
    L.set_edge(o.BOTTOM, o.TRACTION)
    L.set_edge(o.TOP, o.VELOCITY, (0.001, 0.0))
    U0 = smooth_field(nx, ny, seed=4, amp=0.03, periodic=False)
    L.init(U0, None, 2)
    L.step(nsteps)
    U, P, S = L.state()
    return L.populations(), U, P, S, L.displacement(), L.status


def test_results_do_not_depend_on_the_thread_count():
    before = o.threads()
    try:
        ref = _run(1)
        for t in (2, 3, 8):
            got = _run(t)
            for a, b in zip(ref[:5], got[:5]):
                assert np.array_equal(a, b)
            assert got[5] == ref[5]
    finally:
        o.set_threads(before)
