"""Host-side bookkeeping of the sensitivity study (no GPU): the tangent
seeds are the derivatives of the inputs the workload builds from p."""
from __future__ import annotations

import numpy as np

from paper_1606_01805_gb300 import sensitivity as sens
from paper_1606_01805_gb300 import workloads as W


def _inputs(p):
    wl = W.sensitivity_ellipse(*p)
    q = wl.particles[0]
    return np.array([q.dim[0], q.dim[1], q.xc, q.yc, q.theta, q.rho_s]), np.array(wl.wall_u, float)


def test_seeds_are_the_input_derivatives():
    p = np.array([2.3, 31.0, 0.0097])
    seed, dwall = sens.seeds(p[0])
    for k in range(3):
        h = 1e-6 * abs(p[k])
        pp, pm = p.copy(), p.copy()
        pp[k] += h
        pm[k] -= h
        (qp, wp), (qm, wm) = _inputs(pp), _inputs(pm)
        assert np.allclose(seed[k], (qp - qm) / (2 * h), rtol=1e-7, atol=1e-9)
        assert np.allclose(dwall[:, :, k], (wp - wm) / (2 * h), rtol=1e-7, atol=1e-9)


def test_ellipse_keeps_the_circle_area_and_marker_count():
    for ar in (1.5, 2.0, 3.0):
        q = W.sensitivity_ellipse(ar, 30.0, 0.01).particles[0]
        assert abs(q.dim[0] * q.dim[1] - 400.0) < 1e-12
        assert abs(q.dim[0] / q.dim[1] - ar) < 1e-12
        assert q.n_markers == W.SENS_MARKERS
