"""The oracle against values the paper prints for its shear-flow transport
study (section 4, the introduction counted as section 1), read from
tests/golden/shear_transport.txt.  Reading of the set-up's figure: the
reference length L_ref is the circle's diameter, the ellipse's major axis
(aspect ratio 2), the square's side and the equilateral triangle's side;
these are the only common choices that give all three printed area ratios."""
import math
from pathlib import Path

import numpy as np
import pytest

from oracle import oracle as o

GOLDEN = Path(__file__).parent / "golden" / "shear_transport.txt"


def golden():
    out = {}
    for line in GOLDEN.read_text().splitlines():
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        key, value = line.split()[:2]
        out[key] = float(value)
    return out


def printed_digits(value):
    """decimal places of a printed value (0.55 -> 2, 0.5 -> 1, 20 -> 0)"""
    s = repr(value)
    return 0 if value == int(value) else len(s.split(".")[1])


def test_fixture_is_consistent():
    g = golden()
    # Re_p = Re L_ref / H (section 4.1)
    assert g["Re"] / g["H_over_Lref"] == g["Re_p"]
    # half the shear of u = u_max y / H in units of u_max / L_ref
    assert 0.5 / g["H_over_Lref"] == g["half_shear_rate"]


def _ring_area(rb, nb, S):
    """area enclosed by the marker ring from the divergence theorem,
    A = (1/2) sum over markers of S_l (r_l . n_l)"""
    return 0.5 * float(np.sum(S * np.einsum("ij,ij->i", rb, nb)))


def test_particle_areas_match_the_printed_ratios():
    """Section 4.1: with one reference length the ellipse, square and
    triangle enclose 0.5, 1.27 and 0.55 of the circle's area.  Checked on
    the oracle's marker rings (positions, normals and lengths S_l) at the
    paper's resolution, L_ref = 100 lattice units, and on the closed-form
    areas it uses for the mass and inertia."""
    g = golden()
    L = 100.0
    s = o.Sim(300, 300, 0.8)
    shapes = [("circle", o.CIRCLE, (L,)), ("ellipse", o.ELLIPSE, (L, L / 2)),
              ("square", o.SQUARE, (L,)), ("triangle", o.TRIANGLE, (L,))]
    ring, closed = {}, {}
    for k, (name, shape, dim) in enumerate(shapes):
        s.add_particle(shape, dim, 150.0, 150.0)
        rb, nb, S = s.markers(k)
        ring[name] = _ring_area(rb, nb, S)
        closed[name] = s.props(k)[2]
    for name in ("ellipse", "square", "triangle"):
        want = g[f"area_ratio_{name}"]
        d = printed_digits(want)
        for area in (ring, closed):
            assert round(area[name] / area["circle"], d) == want, (name, area[name] / area["circle"])
    # the ring's areas are those of the shapes themselves, not only in ratio
    assert ring["circle"] == pytest.approx(math.pi * L * L / 4, rel=1e-12)
    assert ring["square"] == pytest.approx(L * L, rel=1e-12)
    assert ring["triangle"] == pytest.approx(math.sqrt(3) / 4 * L * L, rel=1e-12)
    assert ring["ellipse"] == pytest.approx(math.pi * L * L / 8, rel=1e-6)


def test_couette_set_up_keeps_the_printed_shear():
    """Sections 4.1-4.2: the lower wall at rest, the upper one at u_max,
    H = 4 L_ref, Re = u_max H / nu = 20, the field started from the planar
    Couette profile.  The oracle keeps (1/2) du_x/dy = 0.125 u_max / L_ref
    at every node after 500 steps (L_ref = 8 lattice units here)."""
    g = golden()
    Lref = 8
    H = int(g["H_over_Lref"]) * Lref
    u_max = 0.05
    nu = u_max * H / g["Re"]
    tau = 3.0 * nu + 0.5
    s = o.Sim(16, H + 1, tau, wall_u=((0, 0), (0, 0), (0.0, 0.0), (u_max, 0.0)), init=o.INIT_COUETTE)
    s.step(500)
    _, ux, uy = s.fields()
    half_shear = 0.5 * np.diff(ux, axis=0) * Lref / u_max
    np.testing.assert_allclose(half_shear, g["half_shear_rate"], atol=1e-12)
    assert np.abs(uy).max() < 1e-14
    # the walls carry the printed boundary speeds
    np.testing.assert_allclose(ux[0], 0.0, atol=1e-14)
    np.testing.assert_allclose(ux[-1], u_max, rtol=1e-12)
