"""Pins of the oracle's tube segment (kind 3: rmin, rmax, dz, sphi, dphi).

Hand-derived closed forms on a quarter wedge (sphi 0, dphi pi/2) and a
three-quarter wedge (dphi 3 pi/2, not convex), the whole turn equal to the
tube (Cauchy's mean chord for a convex segment is in test_oracle_pins.py).
"""
import math

import numpy as np
import pytest

from paper_1312_0816_gb300 import scenes

Q = (0.0, 10.0, 10.0, 0.0, math.pi / 2)          # solid quarter wedge
T = (0.0, 10.0, 10.0, 0.0, 1.5 * math.pi)        # three quarters: all but x > 0, y < 0
S = (4.0, 10.0, 10.0, 0.0, math.pi / 2)          # quarter of a shell


def one(orc, params, x, u, what):
    out = orc.shape(scenes.TUBS, params, [x], [u] if u is not None else None, what)
    if isinstance(out, tuple):
        return float(out[0][0]), int(out[1][0])
    return float(out[0])


@pytest.mark.parametrize("params,x,u,want,face", [
    # enters the quarter wedge through the face at phi = 0 (the plane y = 0, x in [0, 10])
    (Q, (5.0, -20.0, 0.0), (0.0, 1.0, 0.0), 20.0, 8),
    # through the face at phi = pi/2 (x = 0, y in [0, 10])
    (Q, (-20.0, 5.0, 0.0), (1.0, 0.0, 0.0), 20.0, 9),
    # through the curved surface from the wedge's side: x = 6 crosses rho = 10 at y = 8
    (Q, (6.0, 30.0, 0.0), (0.0, -1.0, 0.0), 22.0, 6),
    # moving away in the excluded quadrant
    (Q, (-5.0, -5.0, 0.0), (-1.0, 0.0, 0.0), math.inf, -1),
    # the three-quarter wedge: x = 5 going +y enters at y = 0 (face at phi = 0)
    (T, (5.0, -20.0, 0.0), (0.0, 1.0, 0.0), 20.0, 8),
    # y = -5 going -x enters at x = 0 (face at phi = 3 pi/2: x = 0, y in [-10, 0])
    (T, (20.0, -5.0, 0.0), (-1.0, 0.0, 0.0), 20.0, 9),
    # the shell quarter: the ray x = 2 crosses the plane of the face phi = 0
    # at r = 2 < rmin, in the hole, and enters through the inner surface at
    # y = sqrt(16 - 4)
    (S, (2.0, -20.0, 0.0), (0.0, 1.0, 0.0), 20.0 + math.sqrt(12.0), 7),
    # z-plane entry inside the wedge
    (Q, (3.0, 3.0, 25.0), (0.0, 0.0, -1.0), 15.0, 5),
])
def test_dist_out_closed_form(orc, params, x, u, want, face):
    s, f = one(orc, params, x, u, "dist_out")
    assert s == pytest.approx(want, rel=1e-14, abs=1e-13) if math.isfinite(want) else math.isinf(s)
    assert f == face


@pytest.mark.parametrize("params,x,u,want,face", [
    # from inside the quarter wedge going +y: leaves through rho = 10 at y = sqrt(75)
    (Q, (5.0, 1.0, 0.0), (0.0, 1.0, 0.0), math.sqrt(75.0) - 1.0, 6),
    # going -y: leaves through the face at phi = 0 (y = 0)
    (Q, (5.0, 1.0, 0.0), (0.0, -1.0, 0.0), 1.0, 8),
    # the three-quarter wedge is not convex: from (-5, -1) going +x the track
    # crosses x = 0 at y = -1, where the wedge ends (face at 3 pi/2)
    (T, (-5.0, -1.0, 0.0), (1.0, 0.0, 0.0), 5.0, 9),
    # from (-5, 1) going +x it stays in the wedge (y > 0) until rho = 10
    (T, (-5.0, 1.0, 0.0), (1.0, 0.0, 0.0), 5.0 + math.sqrt(99.0), 6),
])
def test_dist_in_closed_form(orc, params, x, u, want, face):
    s, f = one(orc, params, x, u, "dist_in")
    assert s == pytest.approx(want, rel=1e-14, abs=1e-13)
    assert f == face


def test_contains_and_safety_closed_form(orc):
    assert one(orc, Q, (5.0, 2.0, 3.0), None, "contains") == 1.0
    assert one(orc, Q, (5.0, -2.0, 3.0), None, "contains") == 0.0
    assert one(orc, Q, (0.0, 0.0, 3.0), None, "contains") == 1.0      # the axis belongs to a solid wedge
    assert one(orc, T, (5.0, -2.0, 3.0), None, "contains") == 0.0
    assert one(orc, T, (-5.0, -2.0, 3.0), None, "contains") == 1.0
    # inside: nearest is the face at phi = 0 (y = 0) at distance 2
    assert one(orc, Q, (5.0, 2.0, 3.0), None, "safety_in") == pytest.approx(2.0, abs=1e-14)
    # outside below the x axis: the face at phi = 0 at distance 3
    assert one(orc, Q, (5.0, -3.0, 0.0), None, "safety_out") == pytest.approx(3.0, abs=1e-14)
    # outside in the opposite quadrant: the axis edge of both faces, distance 5
    assert one(orc, Q, (-3.0, -4.0, 0.0), None, "safety_out") == pytest.approx(5.0, abs=1e-14)
    # outside beyond the curved surface inside the wedge: radial distance
    assert one(orc, Q, (12.0, 5.0, 0.0), None, "safety_out") == pytest.approx(3.0, abs=1e-14)
    # the excluded quadrant of the three-quarter wedge: nearest face at distance 2
    assert one(orc, T, (5.0, -2.0, 0.0), None, "safety_out") == pytest.approx(2.0, abs=1e-14)


def test_whole_turn_is_the_tube(orc):
    rng = np.random.default_rng(3)
    x = rng.uniform(-30, 30, size=(20000, 3))
    u = rng.normal(size=(20000, 3))
    u /= np.linalg.norm(u, axis=1, keepdims=True)
    seg = (3.0, 10.0, 10.0, 0.7, 2.0 * math.pi)
    for what in ("dist_out", "dist_in"):
        a, fa = orc.shape(scenes.TUBS, seg, x, u, what)
        b, fb = orc.shape(scenes.TUBE, seg[:3], x, u, what)
        assert np.array_equal(a, b) and np.array_equal(fa, fb)
    for what in ("contains", "safety_out", "safety_in"):
        assert np.array_equal(orc.shape(scenes.TUBS, seg, x, None, what), orc.shape(scenes.TUBE, seg[:3], x, None, what))
