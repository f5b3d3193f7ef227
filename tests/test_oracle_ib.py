"""Pins of the oracle's immersed-boundary and rigid-body half (Sections 2.2
and 2.3): MLS reproduction properties (Eqs. 8-10), the alternative weights
(Eqs. 17-20), force conservation of the spreading (Eq. 12), closed-form
stress integrals (Eqs. 13-14), the two-level rigid-body update (Eqs. 15-16)
and symmetries of the whole coupled step."""
import numpy as np
import pytest

from oracle import oracle as o

from .test_oracle_golden import golden

RNG = np.random.default_rng(777)


def _rand_points(n):
    return 20 + 10 * RNG.random((n, 2))


def test_mls_partition_of_unity_and_linear_reproduction():
    """Linear basis p = (1, x, y) (Eq. 9): the transfer weights sum to one and
    reproduce x and y; the derivative rows reproduce the gradient of any
    linear field."""
    for x, y in _rand_points(200):
        ix, iy, phi = o.mls(x, y)
        assert phi[0].sum() == pytest.approx(1.0, abs=1e-14)
        assert phi[0] @ ix == pytest.approx(x, abs=1e-12)
        assert phi[0] @ iy == pytest.approx(y, abs=1e-12)
        assert abs(phi[1].sum()) < 1e-13 and abs(phi[2].sum()) < 1e-13
        assert phi[1] @ ix == pytest.approx(1.0, abs=1e-12)
        assert abs(phi[1] @ iy) < 1e-12
        assert abs(phi[2] @ ix) < 1e-12
        assert phi[2] @ iy == pytest.approx(1.0, abs=1e-12)


def test_mls_support_is_nearest_three_by_three():
    """The nine nodes are the 3x3 block around the nearest node (Figure 1);
    every normalised distance stays below the cut-off r = 1 of Eq. 10."""
    rmax = 0
    for x, y in _rand_points(500):
        ix, iy, _ = o.mls(x, y)
        i0, j0 = int(np.floor(x + 0.5)), int(np.floor(y + 0.5))
        assert sorted(set(ix.tolist())) == [i0 - 1, i0, i0 + 1]
        assert sorted(set(iy.tolist())) == [j0 - 1, j0, j0 + 1]
        rmax = max(rmax, (np.hypot(ix - x, iy - y) / 2.6).max())
    assert rmax <= np.sqrt(2 * 1.5 ** 2) / 2.6 + 1e-12
    assert rmax < 1


def test_mls_equals_weighted_least_squares_in_global_coordinates():
    """Eq. 9 written with the global basis (1, x, y): minimising J for the unit
    data vectors gives the same phi as the oracle's local-coordinate solve."""
    for x, y in _rand_points(50):
        ix, iy, phi = o.mls(x, y)
        r = np.hypot(ix - x, iy - y) / 2.6
        W = np.exp(-(r / 0.3) ** 2)
        P = np.stack([np.ones(9), ix, iy], axis=1)
        sw = np.sqrt(W)[:, None]
        # phi_k = p(x)^T a_k with a_k the weighted LS fit of the k-th unit vector
        a, *_ = np.linalg.lstsq(sw * P, sw * np.eye(9), rcond=None)
        np.testing.assert_allclose(np.array([1.0, x, y]) @ a, phi[0], atol=1e-11)


def test_mls_on_a_node_is_symmetric():
    """A marker sitting on a node: weights are symmetric under reflections."""
    _, _, phi = o.mls(17.0, 9.0)
    p = phi[0].reshape(3, 3)
    np.testing.assert_allclose(p, p[::-1, :], atol=1e-15)
    np.testing.assert_allclose(p, p[:, ::-1], atol=1e-15)
    np.testing.assert_allclose(p, p.T, atol=1e-15)


def test_exponential_weight_values():
    """Eq. 10 with alpha = 0.3: W(0) = 1, W(0.3) = 1/e, W = 0 beyond r = 1."""
    assert o.weight(o.W_EXP, 0.0) == 1.0
    assert o.weight(o.W_EXP, 0.3) == pytest.approx(np.exp(-1.0), rel=1e-15)
    assert o.weight(o.W_EXP, 1.0 + 1e-9) == 0.0


def test_alternative_weights():
    """Eq. 18 vanishes at r = 1; Eq. 19 as printed is 1/4 there; Eq. 20 read in
    q = 2 r is the 4-point kernel: its integer shifts sum to one."""
    assert o.weight(o.W_QUARTIC, 1.0) == pytest.approx(0.0, abs=1e-15)
    assert o.weight(o.W_QUARTIC, 0.0) == 1.0
    assert o.weight(o.W_COSINE, 1.0) == pytest.approx(0.25, abs=1e-15)
    assert o.weight(o.W_CUBIC, 0.0) == pytest.approx(2 / 3)
    for q in RNG.random(50):
        s = sum(o.weight(o.W_POLY, abs(q - j) / 2) for j in range(-2, 4))
        assert s == pytest.approx(1.0, abs=1e-14)
        even = sum(o.weight(o.W_POLY, abs(q - j) / 2) for j in range(-2, 4, 2))
        assert even == pytest.approx(0.5, abs=1e-14)
    for kind in (o.W_CUBIC, o.W_QUARTIC, o.W_COSINE, o.W_POLY):
        for x, y in _rand_points(20):
            _, _, phi = o.mls(x, y, weight=kind)
            assert phi[0].sum() == pytest.approx(1.0, abs=1e-13)


def _sim_with_circle(R=10.0, n=64, **kw):
    s = o.Sim(80, 60, 0.8, **kw)
    s.add_particle(o.CIRCLE, (2 * R,), 40.3, 30.2, n_markers=n)
    return s


def test_markers_of_shapes():
    """Markers lie on the surface, normals are outward unit vectors, the S_l
    sum to the perimeter; area and inertia follow the closed forms."""
    s = o.Sim(200, 200, 0.8)
    cases = [(o.CIRCLE, (32.0,)), (o.ELLIPSE, (48.0, 24.0)), (o.RECT, (64.0, 16.0)),
             (o.SQUARE, (32.0,)), (o.TRIANGLE, (40.0,))]
    for k, (shape, dim) in enumerate(cases):
        s.add_particle(shape, dim, 100.0, 100.0)
        rb, nb, S = s.markers(k)
        m, I, A = s.props(k)
        np.testing.assert_allclose(np.hypot(nb[:, 0], nb[:, 1]), 1.0, atol=1e-14)
        np.testing.assert_allclose((S[:, None] * nb).sum(0), 0, atol=1e-9)
        assert (np.einsum("ij,ij->i", rb, nb) > 0).all()  # outward (star-shaped about 0)
        if shape == o.CIRCLE:
            np.testing.assert_allclose(np.hypot(*rb.T), 16.0, atol=1e-12)
            assert S.sum() == pytest.approx(np.pi * 32, rel=1e-13)
            assert A == pytest.approx(np.pi * 16 ** 2) and I == pytest.approx(m * 32 ** 2 / 8)
        if shape == o.ELLIPSE:
            np.testing.assert_allclose((rb[:, 0] / 24) ** 2 + (rb[:, 1] / 12) ** 2, 1, atol=1e-12)
            # Ramanujan's second approximation of the perimeter
            a, b = 24.0, 12.0
            h = ((a - b) / (a + b)) ** 2
            P = np.pi * (a + b) * (1 + 3 * h / (10 + np.sqrt(4 - 3 * h)))
            assert S.sum() == pytest.approx(P, rel=1e-9)
            np.testing.assert_allclose(S, S[0], rtol=1e-12)
            # consecutive markers are equally spaced in arc length: chords nearly equal
            ch = np.hypot(*np.diff(np.vstack([rb, rb[:1]]), axis=0).T)
            assert ch.max() / ch.min() < 1.001
            assert A == pytest.approx(np.pi * a * b) and I == pytest.approx(m * (a * a + b * b) / 4)
        if shape == o.RECT:
            assert S.sum() == pytest.approx(2 * (64 + 16), rel=1e-13)
            on_x = np.isclose(np.abs(rb[:, 0]), 32.0)
            on_y = np.isclose(np.abs(rb[:, 1]), 8.0)
            assert (on_x | on_y).all()
            assert I == pytest.approx(m * (64 ** 2 + 16 ** 2) / 12)
        if shape == o.SQUARE:
            assert I == pytest.approx(m * 32 ** 2 / 6)
        if shape == o.TRIANGLE:
            assert S.sum() == pytest.approx(120.0, rel=1e-13)
            assert A == pytest.approx(np.sqrt(3) / 4 * 40 ** 2)
            assert I == pytest.approx(m * 40 ** 2 / 12)
            # distance from centroid to every face is the inradius s / (2 sqrt 3)
            np.testing.assert_allclose(np.einsum("ij,ij->i", rb, nb), 40 / (2 * np.sqrt(3)),
                                       atol=1e-12)
        # spacing close to the 0.3 dx of Sections 3-4
        assert 0.25 < S.mean() < 0.35


def test_spreading_conserves_force_and_torque():
    """Eq. 12 with c_l = S_l: the lattice receives exactly sum_l S_l F_l, and,
    by linear reproduction, the matching moment sum_l S_l x_l x F_l."""
    s = _sim_with_circle()
    s.set_history(0, (40.3, 30.2), 0.3, (0.01, -0.004), 0.002, (40.3, 30.2), 0.3, (0, 0), 0)
    ny, nx = 60, 80
    yy, xx = np.mgrid[0:ny, 0:nx]
    ux = 0.01 * np.sin(0.2 * xx + 0.1 * yy)
    uy = 0.005 * np.cos(0.15 * yy - 0.3 * xx)
    flb, sf, tq = s.spread(0, ux, uy)
    assert np.abs(sf).max() > 1e-3
    np.testing.assert_allclose(flb.reshape(2, -1).sum(1), sf, atol=1e-14)
    lat_tq = (xx * flb[1] - yy * flb[0]).sum()
    assert lat_tq == pytest.approx(tq, rel=1e-11)


def test_marker_force_zero_when_fluid_moves_rigidly():
    """Eq. 11: if the lattice velocity is the body's rigid motion (a linear
    field, reproduced exactly by MLS) the marker forces vanish."""
    s = _sim_with_circle()
    X, U, W = np.array([40.3, 30.2]), np.array([0.01, -0.004]), 0.002
    s.set_history(0, X, 0.3, U, W, X, 0.3, U, W)
    yy, xx = np.mgrid[0:60, 0:80].astype(float)
    ux = U[0] - W * (yy - X[1])
    uy = U[1] + W * (xx - X[0])
    flb, sf, _ = s.spread(0, ux, uy)
    assert np.abs(flb).max() < 1e-15


def _fields(fn):
    yy, xx = np.mgrid[0:60, 0:80].astype(float)
    return fn(xx, yy)


def test_stress_uniform_pressure_gives_no_load():
    """A uniform density has no net force or moment on a closed ring."""
    s = _sim_with_circle()
    rho, ux, uy = _fields(lambda x, y: (np.full_like(x, 1.07), 0 * x, 0 * x))
    F, M = s.stress_force(0, rho, ux, uy)
    assert np.abs(F).max() < 1e-14 and abs(M) < 1e-13


def test_stress_linear_pressure_closed_form():
    """rho = 1 + beta x: p = c_s^2 (rho - 1) is exactly linear at the probes,
    so Eq. 13 gives F_x = -c_s^2 beta pi R (R + 1.2) for equally spaced
    markers on a circle of radius R, and no moment."""
    R, beta = 10.0, 1e-3
    s = _sim_with_circle(R=R)
    rho, ux, uy = _fields(lambda x, y: (1 + beta * (x - 40.3), 0 * x, 0 * x))
    F, M = s.stress_force(0, rho, ux, uy)
    assert F[0] == pytest.approx(-beta / 3 * np.pi * R * (R + 1.2), rel=1e-11)
    assert abs(F[1]) < 1e-14 and abs(M) < 1e-13


def test_stress_linear_velocity_has_no_load():
    """A linear velocity field has a constant symmetric stress: zero net force
    and zero moment on a closed ring."""
    s = _sim_with_circle()
    rho, ux, uy = _fields(lambda x, y: (1 + 0 * x, 1e-3 * (0.3 * x + 0.7 * y), 1e-3 * (-0.2 * x - 0.3 * y)))
    F, M = s.stress_force(0, rho, ux, uy)
    assert np.abs(F).max() < 1e-15 and abs(M) < 1e-14


@pytest.mark.parametrize("rho0", [1.0, 1.3])
def test_stress_potential_vortex_torque(rho0):
    """Potential vortex u_theta = G / r around the particle: tau_r_theta =
    -2 rho nu G / r^2, taken at the probe radius R + 1.2 (Section 2.3), gives
    M = -4 pi rho nu G R^2 / (R + 1.2)^2.  MLS fits the curved field to O(h^2)."""
    R, G, tau = 10.0, 0.05, 0.8
    nu = (tau - 0.5) / 3
    s = _sim_with_circle(R=R)

    def vortex(x, y):
        dx, dy = x - 40.3, y - 30.2
        r2 = np.maximum(dx * dx + dy * dy, 1.0)
        return rho0 + 0 * x, -G * dy / r2, G * dx / r2

    F, M = s.stress_force(0, *_fields(vortex))
    want = -4 * np.pi * rho0 * nu * G * R ** 2 / (R + 1.2) ** 2
    assert M == pytest.approx(want, rel=0.02)
    assert np.abs(F).max() < 1e-3 * abs(want)  # net force only from the O(h^2) fit error


def test_stress_acceleration_correction():
    """p_l = p_P + rho 1.2 (d_t u_l . n_l) with d_t u_l the change of the rigid
    velocity between the stored levels: for a translating circle at rest in
    still fluid, F = -1.2 pi R dU."""
    R = 10.0
    s = _sim_with_circle(R=R)
    X = np.array([40.3, 30.2])
    dU = np.array([2e-4, -1e-4])
    s.set_history(0, X, 0.0, dU, 0.0, X, 0.0, (0, 0), 0.0)
    F, M = s.stress_force(0, *_fields(lambda x, y: (1 + 0 * x, 0 * x, 0 * x)))
    np.testing.assert_allclose(F, -1.2 * np.pi * R * dU, rtol=1e-12)
    assert abs(M) < 1e-15


def test_rigid_update_constant_force():
    """Eqs. 15-16 with a constant acceleration a: the velocity is exactly
    u0 + a n (two-level form exact for linear data, after the one-level
    start); the position error against x0 + u0 n + a n^2/2 is the start-up
    error a/2 propagated by the x-recursion: 3a/4 (1 - 3^-n)."""
    s = o.Sim(200, 200, 0.8, gravity=(0, 0))
    s.add_particle(o.CIRCLE, (20.0,), 100.0, 100.0, rho_s=2.0, u0=(0.01, 0.0), omega0=0.001,
                   n_markers=64)
    m, I, A = s.props(0)
    F = np.array([3e-3, -1e-3])
    Mz = 2e-3
    for n in range(1, 31):
        s.rigid_update(0, F, Mz)
        p = s.particles()[0]
        a = F / m
        al = Mz / I
        assert p["u"][0] == pytest.approx(0.01 + a[0] * n, rel=1e-12)
        assert p["u"][1] == pytest.approx(a[1] * n, rel=1e-12)
        assert p["omega"] == pytest.approx(0.001 + al * n, rel=1e-12)
        corr = 0.75 * (1 - 3.0 ** (-n))
        assert p["xc"] == pytest.approx(100 + 0.01 * n + a[0] * (n * n / 2 + corr), rel=1e-13)
        assert p["yc"] == pytest.approx(100 + a[1] * (n * n / 2 + corr), rel=1e-13)
        assert p["theta"] == pytest.approx(0.001 * n + al * (n * n / 2 + corr), abs=1e-13)


def test_rigid_update_buoyancy():
    """Gravity acts on the particle with its buoyancy: a = (1 - 1/rho_s) g."""
    g = (0.0, -1e-5)
    s = o.Sim(200, 200, 0.8, gravity=g)
    s.add_particle(o.CIRCLE, (20.0,), 100.0, 100.0, rho_s=1.5, n_markers=64)
    s.rigid_update(0, np.zeros(2), 0.0)
    assert s.particles()[0]["u"][1] == pytest.approx((1 - 1 / 1.5) * g[1], rel=1e-14)


def test_particle_at_rest_stays_at_rest():
    """Particle at rest in fluid at rest between walls at rest: nothing moves
    beyond round-off (the weights of Eq. 3 sum to one only to rounding)."""
    s = o.Sim(60, 40, 0.8)
    s.add_particle(o.ELLIPSE, (16.0, 8.0), 30.0, 20.0, theta=0.4)
    s.step(40)
    p = s.particles()[0]
    np.testing.assert_allclose((p["xc"], p["yc"], p["theta"]), (30.0, 20.0, 0.4), atol=1e-14)
    assert max(abs(p["u"][0]), abs(p["u"][1]), abs(p["omega"])) < 1e-15
    _, ux, uy = s.fields()
    assert np.abs(ux).max() < 1e-15 and np.abs(uy).max() < 1e-15


def test_centred_circle_in_antisymmetric_couette_stays_centred():
    """Rotating the channel by pi about the particle centre maps the flow
    onto itself, so a centred circle (even marker count) feels no lift."""
    nx, ny, U = 64, 41, 0.01
    H = ny - 1
    s = o.Sim(nx, ny, 0.8, wall_u=((0, 0), (0, 0), (-U, 0), (U, 0)), init=o.INIT_COUETTE)
    s.add_particle(o.CIRCLE, (12.0,), 31.5, H / 2, n_markers=64)
    s.step(300)
    p = s.particles()[0]
    assert abs(p["yc"] - H / 2) < 1e-12
    assert abs(p["u"][1]) < 1e-14
    assert abs(p["xc"] - 31.5) < 1e-11  # no net drift in x either
    assert p["omega"] < 0  # co-rotates with the shear


def test_mirror_release_positions_give_mirrored_trajectories():
    """Release at y0 and at H - y0 in antisymmetric Couette: the pi-rotation
    maps one run onto the other (y -> H - y, u -> -u, omega -> omega)."""
    nx, ny, U = 64, 41, 0.01
    H = ny - 1
    out = []
    for y0, x0 in ((0.35 * H, 20.0), (0.65 * H, nx - 1 - 20.0)):
        s = o.Sim(nx, ny, 0.8, wall_u=((0, 0), (0, 0), (-U, 0), (U, 0)), init=o.INIT_COUETTE)
        s.add_particle(o.CIRCLE, (10.0,), x0, y0, n_markers=48)
        s.step(200)
        out.append(s.particles()[0])
    a, b = out
    assert a["yc"] + b["yc"] == pytest.approx(H, abs=1e-10)
    assert a["u"][0] == pytest.approx(-b["u"][0], abs=1e-12)
    assert a["u"][1] == pytest.approx(-b["u"][1], abs=1e-12)
    assert a["omega"] == pytest.approx(b["omega"], abs=1e-12)
    assert abs(a["yc"] - 0.35 * H) > 1e-6  # the particle did move laterally


def test_support_leaving_domain_is_an_error():
    """A particle whose probe supports would cross a wall is rejected."""
    s = o.Sim(60, 40, 0.8)
    with pytest.raises(ValueError):
        s.add_particle(o.CIRCLE, (20.0,), 30.0, 11.0)


def test_marker_force_sign_pushes_fluid_with_the_body():
    """Eq. 11 is U_b - U: a body translating at U_b through still fluid
    spreads the total force U_b * perimeter (with c_l = S_l) onto the lattice."""
    s = _sim_with_circle(R=10.0)
    X, U = np.array([40.3, 30.2]), np.array([0.003, -0.002])
    s.set_history(0, X, 0.0, U, 0.0, X, 0.0, U, 0.0)
    z = np.zeros((60, 80))
    flb, sf, _ = s.spread(0, z, z)
    np.testing.assert_allclose(flb.reshape(2, -1).sum(1), U * np.pi * 20.0, rtol=1e-12)


def test_circle_in_couette_rotates_near_half_shear():
    """Section 4.2: a neutrally buoyant circle in Couette flow at Re = 20
    rotates at omega L / u_max = 0.117, close to half the shear rate (0.125;
    both from tests/golden/shear_transport.txt), and is carried at the local
    undisturbed velocity.  400 x 100 channel, walls at +-U, D = 20, released
    at y = 0.3 H (the plain FP64 workload)."""
    g = golden()
    nx, ny, tau = 400, 100, 0.8
    H = ny - 1
    U = 20 * (tau - 0.5) / 3 / H / 2
    s = o.Sim(nx, ny, tau, wall_u=((0, 0), (0, 0), (-U, 0), (U, 0)), init=o.INIT_COUETTE)
    s.add_particle(o.CIRCLE, (20.0,), 200.0, 0.3 * H, n_markers=63)
    s.step(2000)
    p = s.particles()[0]
    half_shear = 0.5 * 2 * U / H
    assert -p["omega"] / half_shear == pytest.approx(g["omega_eq"] / g["half_shear_rate"], abs=0.05)
    u_local = -U + 2 * U * p["yc"] / H
    assert p["u"][0] == pytest.approx(u_local, rel=0.03)
    assert abs(p["u"][1]) < 0.02 * abs(p["u"][0])  # lateral drift is much slower
