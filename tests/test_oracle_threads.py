"""The oracle's OpenMP rows: the lattice loops give the same bits on any
thread count (each row is one thread's, with the same arithmetic), so the
multi-core CPU baseline times the same computation as the single-core one."""
import numpy as np

from oracle import oracle as o
from paper_1606_01805_gb300 import workloads as W


def _run(threads):
    o.set_threads(threads)
    try:
        wl = W.sedimentation("ellipse", steps=0).with_(nx=90, ny=140)
        wl.particles[0] = W.Particle(W.ELLIPSE, (30.0, 15.0), 45.0, 100.0, theta=0.7, rho_s=1.5)
        sim = W.run_with(o.Sim, wl, steps=15)
        return sim.populations(), sim.particles()
    finally:
        o.set_threads(1)


def test_thread_count_does_not_change_the_bits():
    f1, p1 = _run(1)
    f4, p4 = _run(4)
    assert np.array_equal(f1, f4)
    assert p1 == p4
