"""Seeded synthetic workloads shaped like the paper's flows.

This module only describes inputs (lattice sizes, walls, relaxation time,
particle shapes and placements drawn from seeds).  It holds none of the
method's arithmetic and imports nothing from the library or the oracle, so
both the CUDA path and the oracle can be driven from the same description.

Workloads (lattice units, dx = dt = 1, fluid reference density 1):

* ``couette_circle``: the plain method's channel.  400 x 100 nodes,
  periodic x, Zou-He walls at y = 0 and y = H = 99 moving at -U and +U,
  tau = 0.8 (nu = 0.1), Re = 2U H / nu = 20 so U = 0.010101; one neutrally
  buoyant circle D = 20 with 63 markers released at y = 0.3 H with zero
  velocity (Section 4.1 set-up at this size).
* ``sedimentation``: quiescent fluid in a closed 400 x 1200 box (no-slip
  walls on all sides), tau = 0.7, one circle D = 50 (or an ellipse 50 x 25
  tilted 45 degrees) at density ratio 1.5 released at (200, 1100), marker
  spacing 0.3; gravity 1.4e-5 downwards, which gives a terminal Reynolds
  number near 10 from a drag balance with C_d ~ 3 (Section 3 set-up).
* ``couette_shapes``: 1024 x 256 channel, bottom wall at rest, top wall at
  U = Re nu / H with Re = 20, tau = 0.8; one particle per instance from
  circle D32, ellipse 48 x 24, rectangle 64 x 16, square 32, triangle 40,
  y0 ~ U[0.2H, 0.8H] and angle ~ U[0, pi) from seed 2 (Section 4.3 set-up).
* ``batched_screening``: 512 independent Couette channels of uneven sizes
  (nx ~ U{256..1024}, ny ~ U{128..256}, bottom wall at rest, top at
  U = Re nu / H, Re = 20, tau = 0.8), one particle each of a random shape
  of the set, aspect ratio ~ U[1, 4] (ellipse, rectangle), circumscribed
  radius 0.1 H .. 0.2 H, centred in x, y0 uniform between the walls with a
  4-node clearance, angle ~ U[0, pi); seed 3 (the screening use case).
* ``large_couette``: 16384 x 4096 antisymmetric Couette channel (cfg of the
  first workload scaled up) with 64 circles D = 20 on a seeded jittered
  grid: a lattice well beyond the 129 MB L2 for the bandwidth roofline.
* ``sensitivity_ellipse`` / ``sensitivity_batch``: the first workload with
  an ellipse of the circle's area, parameterised by aspect ratio, initial
  height and wall speed; 64 seeded parameter triples (seed 4).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field, replace

import numpy as np

PERIODIC, VELOCITY = 0, 1
REST, COUETTE, TAYLOR_GREEN = 0, 1, 2
CIRCLE, ELLIPSE, RECT, SQUARE, TRIANGLE = range(5)
SHAPE_NAMES = {CIRCLE: "circle", ELLIPSE: "ellipse", RECT: "rectangle", SQUARE: "square",
               TRIANGLE: "triangle"}


@dataclass
class Particle:
    shape: int
    dim: tuple
    xc: float
    yc: float
    theta: float = 0.0
    rho_s: float = 1.0
    u0: tuple = (0.0, 0.0)
    omega0: float = 0.0
    n_markers: int = 0

    def kwargs(self):
        return dict(shape=self.shape, dim=tuple(self.dim), xc=self.xc, yc=self.yc,
                    theta=self.theta, rho_s=self.rho_s, u0=tuple(self.u0), omega0=self.omega0,
                    n_markers=self.n_markers)


@dataclass
class Workload:
    name: str
    nx: int
    ny: int
    tau: float
    bc: tuple = (PERIODIC, PERIODIC, VELOCITY, VELOCITY)
    wall_u: tuple = ((0.0, 0.0), (0.0, 0.0), (0.0, 0.0), (0.0, 0.0))
    body_force: tuple = (0.0, 0.0)
    gravity: tuple = (0.0, 0.0)
    init: int = REST
    init_u: float = 0.0
    weight: int = 0
    spacing: float = 0.3
    steps: int = 1000
    particles: list = field(default_factory=list)

    @property
    def cells(self):
        return self.nx * self.ny

    def lattice_kwargs(self):
        return dict(bc=self.bc, wall_u=self.wall_u, body_force=self.body_force,
                    gravity=self.gravity, init=self.init, init_u=self.init_u, weight=self.weight)

    def with_(self, **kw):
        return replace(self, **kw)


def couette_circle(steps=2000):
    nx, ny, tau = 400, 100, 0.8
    H = ny - 1
    nu = (tau - 0.5) / 3.0
    U = 20.0 * nu / H / 2.0
    return Workload("couette_circle_400x100", nx, ny, tau,
                    wall_u=((0, 0), (0, 0), (-U, 0.0), (U, 0.0)), init=COUETTE, steps=steps,
                    particles=[Particle(CIRCLE, (20.0,), 200.0, 0.3 * H, n_markers=63)])


def sedimentation(shape="circle", steps=20000):
    nx, ny = 400, 1200
    p = (Particle(CIRCLE, (50.0,), 200.0, 1100.0, rho_s=1.5) if shape == "circle" else
         Particle(ELLIPSE, (50.0, 25.0), 200.0, 1100.0, theta=math.pi / 4, rho_s=1.5))
    return Workload(f"sedimentation_{shape}_400x1200", nx, ny, 0.7,
                    bc=(VELOCITY,) * 4, gravity=(0.0, -1.4e-5), init=REST, steps=steps,
                    particles=[p])


SHAPE_SET = [(CIRCLE, (32.0,)), (ELLIPSE, (48.0, 24.0)), (RECT, (64.0, 16.0)), (SQUARE, (32.0,)),
             (TRIANGLE, (40.0,))]


def couette_shapes(steps=50000, seed=2):
    nx, ny, tau = 1024, 256, 0.8
    H = ny - 1
    U = 20.0 * (tau - 0.5) / 3.0 / H
    rng = np.random.default_rng(seed)
    out = []
    for shape, dim in SHAPE_SET:
        y0 = float(rng.uniform(0.2 * H, 0.8 * H))
        th = float(rng.uniform(0.0, math.pi))
        out.append(Workload(f"couette_{SHAPE_NAMES[shape]}_1024x256", nx, ny, tau,
                            wall_u=((0, 0), (0, 0), (0.0, 0.0), (U, 0.0)), init=COUETTE,
                            steps=steps, particles=[Particle(shape, dim, nx / 2, y0, theta=th)]))
    return out


def large_couette(nx=16384, ny=4096, n_particles=64, seed=5, steps=100):
    tau = 0.8
    H = ny - 1
    U = 20.0 * (tau - 0.5) / 3.0 / 99.0 / 2.0  # wall speed of the 400 x 100 channel
    rng = np.random.default_rng(seed)
    side = int(round(math.sqrt(n_particles)))
    parts = []
    for k in range(n_particles):
        i, j = k % side, k // side
        x = (i + 0.5 + rng.uniform(-0.2, 0.2)) * nx / side
        y = (j + 0.5 + rng.uniform(-0.2, 0.2)) * H / side
        parts.append(Particle(CIRCLE, (20.0,), float(x), float(y), n_markers=63))
    return Workload(f"large_couette_{nx}x{ny}", nx, ny, tau,
                    wall_u=((0, 0), (0, 0), (-U, 0.0), (U, 0.0)), init=COUETTE, steps=steps,
                    particles=parts)


def shape_for(shape, rc, ar):
    """dims of `shape` with circumscribed radius rc and aspect ratio ar"""
    if shape == CIRCLE:
        return (2 * rc,)
    if shape == ELLIPSE:
        return (2 * rc, 2 * rc / ar)
    if shape == RECT:
        w = 2 * rc * ar / math.sqrt(1 + ar * ar)
        return (w, w / ar)
    if shape == SQUARE:
        return (2 * rc / math.sqrt(2),)
    return (rc * math.sqrt(3),)


def batched_screening(n=512, seed=3, nx_range=(256, 1024), ny_range=(128, 256), steps=10000,
                      tau=0.8):
    rng = np.random.default_rng(seed)
    out = []
    for k in range(n):
        nx = int(rng.integers(nx_range[0], nx_range[1] + 1))
        ny = int(rng.integers(ny_range[0], ny_range[1] + 1))
        H = ny - 1
        U = 20.0 * (tau - 0.5) / 3.0 / H
        shape = int(rng.integers(0, 5))
        ar = float(rng.uniform(1.0, 4.0))
        rc = float(rng.uniform(0.1, 0.2)) * H
        th = float(rng.uniform(0.0, math.pi))
        y0 = float(rng.uniform(rc + 4.0, H - rc - 4.0))
        out.append(Workload(f"screen_{k}_{SHAPE_NAMES[shape]}_{nx}x{ny}", nx, ny, tau,
                            wall_u=((0, 0), (0, 0), (0.0, 0.0), (U, 0.0)), init=COUETTE,
                            steps=steps,
                            particles=[Particle(shape, shape_for(shape, rc, ar), nx / 2, y0,
                                                theta=th)]))
    return out


SENS_MARKERS = 72  # fixed marker count of the sensitivity ellipses (spacing <= 1.05 up to AR 3)


def sensitivity_ellipse(ar, y0, U, steps=2000, theta=0.0, nx=400, ny=100, tau=0.8):
    """The plain method's channel (``couette_circle``) with the circle
    replaced by an ellipse of aspect ratio `ar` and the area of the D = 20
    circle (semi-axes 10 sqrt(ar) and 10 / sqrt(ar)), released at y0 with
    angle theta; walls at -U and +U.  The three parameters (ar, y0, U) are
    the inputs of the sensitivity study; the marker count is fixed."""
    a, b = 10.0 * math.sqrt(ar), 10.0 / math.sqrt(ar)
    return Workload(f"sens_ellipse_ar{ar:.4f}_{nx}x{ny}", nx, ny, tau,
                    wall_u=((0, 0), (0, 0), (-U, 0.0), (U, 0.0)), init=COUETTE, steps=steps,
                    particles=[Particle(ELLIPSE, (2 * a, 2 * b), nx / 2, y0, theta=theta,
                                        n_markers=SENS_MARKERS)])


def sensitivity_batch(n=64, seed=4, steps=2000):
    """n seeded parameter triples (ar ~ U[1.5, 3], y0 ~ U[0.25 H, 0.4 H],
    U ~ U0 * U[0.8, 1.2] with U0 the wall speed of Re = 20) and angles
    ~ U[0, pi), as an [n][3] array and the angles."""
    tau, H = 0.8, 99.0
    U0 = 20.0 * (tau - 0.5) / 3.0 / H / 2.0
    rng = np.random.default_rng(seed)
    P = np.stack([rng.uniform(1.5, 3.0, n), rng.uniform(0.25 * H, 0.4 * H, n),
                  U0 * rng.uniform(0.8, 1.2, n)], axis=1)
    th = rng.uniform(0.0, math.pi, n)
    return P, th


def batch_config(wl: Workload):
    """make_config keyword arguments of one instance of a batch"""
    return dict(nx=wl.nx, ny=wl.ny, tau=wl.tau, **wl.lattice_kwargs())


def random_populations(nx, ny, seed, base, amp=0.02, smooth=0.05):
    """Seeded positive populations [9][ny][nx] around the caller's 9-vector
    `base`: base_i * (1 + amp * white noise + smooth * a random smooth field
    per direction), the latter giving the lattice a smooth momentum field."""
    rng = np.random.default_rng(seed)
    base = np.asarray(base, dtype=np.float64).reshape(9, 1, 1)
    yy, xx = np.mgrid[0:ny, 0:nx]
    ph = rng.uniform(0, 2 * np.pi, (9, 2))
    kx = rng.integers(1, 3, 9)
    ky = rng.integers(1, 3, 9)
    sm = np.stack([np.sin(2 * np.pi * kx[i] * xx / nx + ph[i, 0]) *
                   np.cos(2 * np.pi * ky[i] * yy / ny + ph[i, 1]) for i in range(9)])
    return base * (1 + amp * rng.uniform(-1, 1, (9, ny, nx)) + smooth * sm)


def run_with(sim_factory, wl: Workload, steps=None, populations=None):
    """Create a simulation through `sim_factory(nx, ny, tau, **lattice_kwargs)`,
    add the workload's particles and advance `steps` (default: wl.steps)."""
    sim = sim_factory(wl.nx, wl.ny, wl.tau, **wl.lattice_kwargs())
    if populations is not None:
        sim.set_populations(populations)
    for p in wl.particles:
        sim.add_particle(**p.kwargs())
    n = wl.steps if steps is None else steps
    if n:
        sim.step(n)
    return sim
