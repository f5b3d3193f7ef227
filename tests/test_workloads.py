"""The seeded synthetic inputs: every workload has the sizes, wall speeds,
particles and parameter ranges its recipe states, is reproducible from its
seed, and keeps every particle's MLS support inside its lattice."""
import math

import numpy as np
import pytest

from paper_1606_01805_gb300 import workloads as W


def _re(wl, u_rel):
    """Reynolds number u_rel H / nu with H = ny - 1 and nu = (tau - 1/2) / 3"""
    return u_rel * (wl.ny - 1) / ((wl.tau - 0.5) / 3.0)


def _circumradius(p):
    d = p.dim
    if p.shape == W.CIRCLE:
        return d[0] / 2
    if p.shape == W.ELLIPSE:
        return d[0] / 2
    if p.shape == W.RECT:
        return math.hypot(d[0], d[1]) / 2
    if p.shape == W.SQUARE:
        return d[0] / math.sqrt(2)
    return d[0] / math.sqrt(3)


def _support_inside(wl):
    """every particle's circumscribed circle plus the probe distance (1.2)
    and the 3 x 3 support (1.5) stays off the y walls"""
    for p in wl.particles:
        r = _circumradius(p) + 1.2 + 1.5
        assert r < p.yc < wl.ny - 1 - r, (wl.name, p)


def test_plain_channel():
    wl = W.couette_circle()
    assert (wl.nx, wl.ny, wl.tau) == (400, 100, 0.8)
    (_, _), (_, _), (ub, _), (ut, _) = wl.wall_u
    assert ub == -ut and _re(wl, ut - ub) == pytest.approx(20.0)
    (p,) = wl.particles
    assert (p.shape, p.dim, p.xc, p.n_markers) == (W.CIRCLE, (20.0,), 200.0, 63)
    assert p.yc == pytest.approx(0.3 * 99)
    _support_inside(wl)


@pytest.mark.parametrize("shape", ["circle", "ellipse"])
def test_sedimentation_box(shape):
    wl = W.sedimentation(shape)
    assert (wl.nx, wl.ny, wl.tau) == (400, 1200, 0.7)
    assert wl.bc == (W.VELOCITY,) * 4 and all(u == (0, 0) or u == (0.0, 0.0) for u in wl.wall_u)
    assert wl.gravity == (0.0, -1.4e-5)
    (p,) = wl.particles
    assert (p.xc, p.yc, p.rho_s) == (200.0, 1100.0, 1.5)
    if shape == "circle":
        assert p.dim == (50.0,)
    else:
        assert p.dim == (50.0, 25.0) and p.theta == pytest.approx(math.pi / 4)


def test_shape_set():
    wls = W.couette_shapes()
    assert [w.particles[0].shape for w in wls] == [W.CIRCLE, W.ELLIPSE, W.RECT, W.SQUARE, W.TRIANGLE]
    for w in wls:
        assert (w.nx, w.ny, w.tau) == (1024, 256, 0.8)
        (_, _), (_, _), (ub, _), (ut, _) = w.wall_u
        assert ub == 0.0 and _re(w, ut) == pytest.approx(20.0)
        p = w.particles[0]
        assert 0.2 * 255 <= p.yc <= 0.8 * 255 and 0.0 <= p.theta < math.pi
        _support_inside(w)
    again = W.couette_shapes()
    assert [w.particles[0].kwargs() for w in wls] == [w.particles[0].kwargs() for w in again]


def test_large_lattice():
    wl = W.large_couette()
    assert (wl.nx, wl.ny, len(wl.particles)) == (16384, 4096, 64)
    ch = W.couette_circle()
    assert wl.wall_u == ch.wall_u  # the plain channel's wall speeds
    assert all(p.dim == (20.0,) and p.n_markers == 63 for p in wl.particles)
    assert all(0 < p.xc < wl.nx for p in wl.particles)
    _support_inside(wl)
    # bodies are far apart: a regular 8 x 8 grid (spacing nx / 8 by H / 8)
    # jittered by at most 0.2 of a spacing, so centres are at least 0.6 H / 8
    # apart, far beyond the bodies' supports
    xy = np.array([(p.xc, p.yc) for p in wl.particles])
    d = np.hypot(*(xy[:, None, :] - xy[None, :, :]).transpose(2, 0, 1))
    assert d[~np.eye(64, dtype=bool)].min() >= 0.6 * (wl.ny - 1) / 8


def test_screening_batch():
    wls = W.batched_screening(steps=0)
    assert len(wls) == 512
    nx = np.array([w.nx for w in wls])
    ny = np.array([w.ny for w in wls])
    assert nx.min() >= 256 and nx.max() <= 1024 and ny.min() >= 128 and ny.max() <= 256
    assert sum(w.cells for w in wls) == 63_343_025
    assert {w.particles[0].shape for w in wls} == set(range(5))
    for w in wls:
        H = w.ny - 1
        (_, _), (_, _), (ub, _), (ut, _) = w.wall_u
        assert ub == 0.0 and _re(w, ut) == pytest.approx(20.0)
        p = w.particles[0]
        assert 0.1 * H - 1e-9 <= _circumradius(p) <= 0.2 * H + 1e-9
        assert p.xc == w.nx / 2
        _support_inside(w)
    again = W.batched_screening(steps=0)
    assert [(w.nx, w.ny, w.particles[0].kwargs()) for w in wls] == \
        [(w.nx, w.ny, w.particles[0].kwargs()) for w in again]


def test_sensitivity_batch():
    P, th = W.sensitivity_batch()
    assert P.shape == (64, 3) and th.shape == (64,)
    H = 99.0
    U0 = 20.0 * (0.8 - 0.5) / 3.0 / H / 2.0
    assert (P[:, 0] >= 1.5).all() and (P[:, 0] <= 3.0).all()
    assert (P[:, 1] >= 0.25 * H).all() and (P[:, 1] <= 0.4 * H).all()
    assert (P[:, 2] >= 0.8 * U0).all() and (P[:, 2] <= 1.2 * U0).all()
    assert (th >= 0).all() and (th < math.pi).all()
    P2, th2 = W.sensitivity_batch()
    assert (P == P2).all() and (th == th2).all()
    for b in range(64):
        wl = W.sensitivity_ellipse(*P[b], theta=float(th[b]))
        _support_inside(wl)
