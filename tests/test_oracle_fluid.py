"""Pins of the oracle's fluid half (Section 2.1) against what the paper and
the mathematics fix: D2Q9 isotropy, the moments of the equilibrium (Eq. 2),
conservation by the forced collision (Eqs. 4-7), the Zou-He wall velocity,
and the analytic Couette, Poiseuille and Taylor-Green solutions."""
import itertools

import numpy as np
import pytest

from oracle import oracle as o

RNG = np.random.default_rng(12345)
D = np.eye(2)


def test_lattice_isotropy():
    """Eq. 3 and its weights: the moments of w_i up to fourth order are those of
    a Gaussian with c_s^2 = 1/3 (the reason the Hermite quadrature works)."""
    e, w = o.lattice()
    e = e.astype(float)
    assert w.sum() == pytest.approx(1.0, abs=1e-15)
    np.testing.assert_allclose(w @ e, 0, atol=1e-15)
    np.testing.assert_allclose(np.einsum("i,ia,ib->ab", w, e, e), D / 3, atol=1e-15)
    np.testing.assert_allclose(np.einsum("i,ia,ib,ic->abc", w, e, e, e), 0, atol=1e-15)
    m4 = np.einsum("i,ia,ib,ic,id->abcd", w, e, e, e, e)
    want = (np.einsum("ab,cd->abcd", D, D) + np.einsum("ac,bd->abcd", D, D)
            + np.einsum("ad,bc->abcd", D, D)) / 9
    np.testing.assert_allclose(m4, want, atol=1e-15)
    speeds = sorted(np.round(np.hypot(e[:, 0], e[:, 1]), 12))
    assert speeds == [0] + [1] * 4 + [round(np.sqrt(2), 12)] * 4
    # the rest population first, then axes, then diagonals; opposites present
    assert tuple(e[0]) == (0, 0)
    for i in range(1, 9):
        assert any((e[j] == -e[i]).all() for j in range(9))


def test_equilibrium_moments():
    """Moments of f^eq (Eq. 2) are rho, rho u and rho (c_s^2 I + u u) exactly."""
    e, _ = o.lattice()
    e = e.astype(float)
    for _ in range(20):
        rho = 0.8 + 0.4 * RNG.random()
        u = 0.1 * (RNG.random(2) - 0.5)
        f = o.feq(rho, *u)
        assert f.sum() == pytest.approx(rho, rel=1e-14)
        np.testing.assert_allclose(f @ e, rho * u, atol=1e-15)
        np.testing.assert_allclose(np.einsum("i,ia,ib->ab", f, e, e),
                                   rho * (D / 3 + np.outer(u, u)), atol=1e-15)


def test_guo_term_moments():
    """Eq. 5: zeroth moment 0, first (1-1/2tau) F, second (1-1/2tau)(uF+Fu)."""
    e, _ = o.lattice()
    e = e.astype(float)
    for _ in range(20):
        tau = 0.55 + RNG.random()
        u = 0.1 * (RNG.random(2) - 0.5)
        F = 1e-3 * (RNG.random(2) - 0.5)
        Fi = o.guo_term(*u, tau, *F)
        k = 1 - 1 / (2 * tau)
        assert abs(Fi.sum()) < 1e-18
        np.testing.assert_allclose(Fi @ e, k * F, atol=1e-18)
        np.testing.assert_allclose(np.einsum("i,ia,ib->ab", Fi, e, e),
                                   k * (np.outer(u, F) + np.outer(F, u)), atol=1e-18)


def test_collision_conserves_mass_and_adds_force():
    """Eq. 4 with Eqs. 6-7: sum f* = sum f and sum f* e = sum f e + F."""
    e, _ = o.lattice()
    e = e.astype(float)
    for _ in range(20):
        f = o.feq(1.0 + 0.05 * RNG.random(), *(0.05 * (RNG.random(2) - 0.5)))
        f = f * (1 + 0.05 * (RNG.random(9) - 0.5))
        F = 1e-3 * (RNG.random(2) - 0.5)
        tau = 0.55 + RNG.random()
        fs = o.collide(f, tau, *F)
        assert fs.sum() == pytest.approx(f.sum(), rel=1e-15)
        np.testing.assert_allclose(fs @ e, f @ e + F, atol=1e-16)


def test_collision_tau_one_is_equilibrium():
    """With tau = 1 and no force Eq. 1 replaces f by f^eq of its own moments."""
    e, _ = o.lattice()
    e = e.astype(float)
    f = o.feq(1.02, 0.03, -0.01) * (1 + 0.1 * (RNG.random(9) - 0.5))
    rho = f.sum()
    u = (f @ e) / rho
    np.testing.assert_allclose(o.collide(f, 1.0), o.feq(rho, *u), atol=1e-16)


def test_couette_is_exact():
    """Planar Couette (Section 4.1): the linear profile between Zou-He walls
    moving at +-U is a steady state that 2000 steps keep to round-off."""
    nx, ny, U = 40, 33, 0.0101
    s = o.Sim(nx, ny, 0.8, wall_u=((0, 0), (0, 0), (-U, 0), (U, 0)), init=o.INIT_COUETTE)
    s.step(2000)
    rho, ux, uy = s.fields()
    y = np.arange(ny)
    want = -U + 2 * U * y / (ny - 1)
    assert np.abs(ux - want[:, None]).max() < 1e-13
    assert np.abs(uy).max() < 1e-14
    assert np.abs(rho - 1).max() < 1e-12


def test_poiseuille_is_exact():
    """Force-driven channel: with the wall reading (forced velocity = wall
    velocity) the parabola u = g y (H - y) / (2 nu) is reproduced to round-off
    (nu = c_s^2 (tau - 1/2))."""
    ny, g = 17, 1e-6
    H = ny - 1
    for tau in (1.0, 0.8):
        s = o.Sim(4, ny, tau, body_force=(g, 0))
        s.step(30000)
        rho, ux, uy = s.fields()
        nu = (tau - 0.5) / 3
        y = np.arange(ny)
        want = g * y * (H - y) / (2 * nu)
        assert np.abs(ux[:, 0] - want).max() / want.max() < 1e-9
        assert np.abs(uy).max() < 1e-15


def test_poiseuille_wrong_viscosity_reading_fails():
    """The printed nu = (2 tau - 1)/c_s^2 would predict a profile 18x smaller:
    the simulated one rules it out."""
    ny, g, tau = 17, 1e-6, 1.0
    s = o.Sim(4, ny, tau, body_force=(g, 0))
    s.step(30000)
    _, ux, _ = s.fields()
    nu_printed = (2 * tau - 1) * 3
    H = ny - 1
    want = g * (H / 2) ** 2 / (2 * nu_printed)
    assert ux[H // 2, 0] > 10 * want


def test_taylor_green_decay():
    """Periodic Taylor-Green vortex: the velocity decays as exp(-2 nu k^2 t)."""
    n, U0, tau = 64, 0.01, 0.8
    nu = (tau - 0.5) / 3
    s = o.Sim(n, n, tau, bc=(0, 0, 0, 0), init=o.INIT_TAYLOR_GREEN, init_u=U0)
    _, ux0, uy0 = s.fields()
    s.step(1000)
    _, ux, uy = s.fields()
    ratio = ((ux * ux0).sum() + (uy * uy0).sum()) / ((ux0 ** 2).sum() + (uy0 ** 2).sum())
    k = 2 * np.pi / n
    assert ratio == pytest.approx(np.exp(-2 * nu * k * k * 1000), rel=1e-3)


@pytest.mark.parametrize("gf", [(0.0, 0.0), (2e-6, -1e-6)])
def test_zou_he_walls_impose_velocity(gf):
    """Zou-He completion: on every wall node of a closed box the forced
    velocity (Eq. 7, constant body force) equals the wall's; corners take
    the velocity of the wall along y and the density of the diagonal
    neighbour."""
    nx, ny = 13, 11
    uw = ((0.0, 0.004), (0.0, -0.003), (0.005, 0.0), (-0.006, 0.0))
    s = o.Sim(nx, ny, 0.7, bc=(1, 1, 1, 1), wall_u=uw, body_force=gf)
    e, _ = o.lattice()
    f = np.stack([np.full((ny, nx), v) for v in o.feq(1.0, 0.0, 0.0)])
    f *= 1 + 0.02 * (RNG.random(f.shape) - 0.5)
    s.set_populations(f)
    rho, ux, uy = s.fields()
    sides = {"left": (slice(1, ny - 1), 0, 0), "right": (slice(1, ny - 1), nx - 1, 1),
             "bottom": (0, slice(1, nx - 1), 2), "top": (ny - 1, slice(1, nx - 1), 3)}
    for name, (ys, xs, k) in sides.items():
        np.testing.assert_allclose(ux[ys, xs], uw[k][0], atol=1e-16, err_msg=name)
        np.testing.assert_allclose(uy[ys, xs], uw[k][1], atol=1e-16, err_msg=name)
    for (y, x, k, dy, dx) in [(0, 0, 2, 1, 1), (0, nx - 1, 2, 1, -1), (ny - 1, 0, 3, -1, 1),
                              (ny - 1, nx - 1, 3, -1, -1)]:
        assert ux[y, x] == pytest.approx(uw[k][0], abs=1e-16)
        assert uy[y, x] == pytest.approx(uw[k][1], abs=1e-16)
        assert rho[y, x] == pytest.approx(rho[y + dy, x + dx], rel=1e-15)


def test_periodic_mass_conservation():
    """Fully periodic lattice with no force: total mass is an invariant."""
    n = 24
    s = o.Sim(n, n, 0.6, bc=(0, 0, 0, 0))
    f = np.stack([np.full((n, n), v) for v in o.feq(1.0, 0.0, 0.0)])
    f *= 1 + 0.05 * (RNG.random(f.shape) - 0.5)
    s.set_populations(f)
    m0 = f.sum()
    s.step(50)
    assert s.populations().sum() == pytest.approx(m0, rel=1e-13)
