"""Oracle runs for the central finite differences of the sensitivity tests
(one process per run; started with the `spawn` method).  Imports the
oracle and the input description only."""
from __future__ import annotations

import math

import numpy as np

from oracle import oracle as o
from paper_1606_01805_gb300 import workloads as W

PROBE = 1.2  # probe distance along the outward normal (Section 2.3)


def oracle_run(args):
    """(final y, mean omega, support trace) of the FP64 oracle for one
    parameter triple.  The trace holds, per step, the nearest node
    (floor(x + 1/2)) of every marker and every probe point of the body
    after the step: a change between two runs is a switch of the 3x3 MLS
    support, where the discrete map is discontinuous."""
    ar, y0, U, theta, steps = args
    wl = W.sensitivity_ellipse(ar, y0, U, steps=steps, theta=theta)
    sim = W.run_with(o.Sim, wl, steps=0)
    rb, nb, _ = sim.markers(0)
    wsum = 0.0
    trace = np.empty((steps, 2 * len(rb), 2), dtype=np.int32)
    for s in range(steps):
        sim.step(1)
        p = sim.particles()[0]
        wsum += p["omega"]
        c, sn = math.cos(p["theta"]), math.sin(p["theta"])
        R = np.array([[c, -sn], [sn, c]])
        xm = np.array([p["xc"], p["yc"]]) + rb @ R.T
        xp = xm + PROBE * (nb @ R.T)
        trace[s] = np.floor(np.concatenate([xm, xp]) + 0.5).astype(np.int32)
    p = sim.particles()[0]
    return p["yc"], wsum / steps, trace
