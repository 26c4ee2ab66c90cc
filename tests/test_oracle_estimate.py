"""Pins of the oracle's under-estimating safety (the cheaper, ROOT-style mode:
every solid replaced by a simpler bound of its distance).

Fixed by the exact safety (pinned on its own in test_oracle_pins.py and
test_oracle_bruteforce.py): never above it; equal to it where every solid's
bound is exact (boxes and tubes, the inside of box, tube and cone mothers);
hand-derived values where the bound is not exact (a cone's supporting
half-planes, a tube segment's whole tube, a polycone's enclosing tube).
"""
import math

import numpy as np
import pytest

from helpers import tracks_from
from paper_1312_0816_gb300 import scenes

ALL = [("box4", 0), ("toy40", 1), ("toy8", 1), ("diff3", None), ("seg4", None), ("pcon4", None), ("pconm", None)]


def _scene(name, seed):
    return scenes.SCENES[name]() if seed is None else scenes.SCENES[name](seed)


@pytest.mark.parametrize("name,seed", ALL)
def test_never_above_the_exact_safety(orc, name, seed):
    sc = _scene(name, seed)
    tr = scenes.sample_tracks(sc, 20000, 51, exclusive=False)
    est = orc.safety_estimate(sc, tr, nthreads=8)
    exact = orc.safety(sc, tr, nthreads=8)
    assert np.all(est >= 0.0)
    # the two formulas round differently: a few ulps of the extent
    assert np.all(est <= exact + 1e-12 * (1.0 + exact))
    if sc.mother_kind == scenes.TUBS:
        assert np.all(est == 0.0)     # such a mother has no bound
    else:
        assert np.mean(est > 0.0) > 0.3


def test_exact_where_every_bound_is_exact(orc):
    """box4 holds only boxes in a box: the estimate is the exact safety, bit
    for bit."""
    sc = scenes.box4(0)
    tr = scenes.sample_tracks(sc, 50000, 52, exclusive=False)
    assert np.array_equal(orc.safety_estimate(sc, tr), orc.safety(sc, tr))


def test_toy_detector_exact_unless_a_cone_is_nearest(orc):
    """toy40: boxes, tube shells and the tube mother have exact bounds; the
    estimate may fall short of the exact safety only where a cone's half-plane
    bound is the smallest, and there it is that cone's bound."""
    sc = scenes.toy40(1)
    tr = scenes.sample_tracks(sc, 30000, 53)
    est = orc.safety_estimate(sc, tr, nthreads=8)
    exact = orc.safety(sc, tr, nthreads=8)
    short = est < exact - 1e-12 * (1.0 + exact)
    assert 0.0 < short.mean() < 0.5
    # removing the cones makes the estimate exact
    keep = sc.kinds != scenes.CONE
    nocone = scenes.Scene("nocone", sc.mother_kind, sc.mother_params, sc.kinds[keep], sc.params[keep], sc.rot[keep],
                          sc.trans[keep])
    assert np.allclose(orc.safety_estimate(nocone, tr), orc.safety(nocone, tr), rtol=1e-13, atol=1e-12)


def _one(orc, mother, daughters, p):
    from helpers import scene_from_spec

    sc = scene_from_spec(mother, daughters, name="est")
    tr = tracks_from(np.array([p], float), np.array([[1.0, 0.0, 0.0]]))
    return float(orc.safety_estimate(sc, tr)[0]), float(orc.safety(sc, tr)[0])


BIG = (0, (500.0, 500.0, 500.0))
EYE = np.eye(3).reshape(9)


def test_cone_half_planes(orc):
    """Cone dz 10, outer radius 5 -> 10, solid, at the origin.  Beside the
    slanted surface the supporting line is the nearest feature: the estimate
    equals the exact distance (20 - 7.5) / sqrt(1 + 1/16); beyond its rim at
    (10, 10) the largest half-plane distance is the z-slab's 30 - 10 = 20, and
    the circumscribed sphere (radius sqrt(200)) gives more, sqrt(1300) -
    sqrt(200), still short of the rim's sqrt(10^2 + 20^2)."""
    cone = (2, (10.0, 0.0, 5.0, 0.0, 10.0), EYE, (0.0, 0.0, 0.0))
    e, x = _one(orc, BIG, [cone], (20.0, 0.0, 0.0))
    assert e == pytest.approx(12.5 / math.sqrt(1.0625), rel=1e-14) and x == pytest.approx(e, rel=1e-14)
    e, x = _one(orc, BIG, [cone], (20.0, 0.0, 30.0))
    assert e == pytest.approx(math.sqrt(1300.0) - math.sqrt(200.0), rel=1e-14)
    assert x == pytest.approx(math.sqrt(500.0), rel=1e-14)


def test_tube_segment_whole_tube(orc):
    """A quarter wedge (r 0..10, dz 10, azimuths 0..pi/2): from (-5, -5, 0), in
    the excluded quadrant inside the whole tube, the estimate is 0; the exact
    distance is to the axis edge, 5 sqrt(2)."""
    seg = (3, (0.0, 10.0, 10.0, 0.0, math.pi / 2), EYE, (0.0, 0.0, 0.0))
    e, x = _one(orc, BIG, [seg], (-5.0, -5.0, 0.0))
    assert e == 0.0 and x == pytest.approx(5.0 * math.sqrt(2.0), rel=1e-14)
    e, x = _one(orc, BIG, [seg], (-20.0, 0.0, 0.0))
    assert e == pytest.approx(10.0, rel=1e-15) and x == pytest.approx(20.0, rel=1e-15)


def test_polycone_enclosing_tube(orc):
    """The bobbin (flanges r 25, waist r 10, z -30..30): from (20, 0, 0) the
    enclosing tube holds the point (estimate 0) while the waist is 10 away;
    from (40, 0, 0) the tube's 15 is short of the flange rim's
    sqrt(15^2 + 25^2)."""
    sc = scenes._scene("b", scenes.BOX, (500.0, 500.0, 500.0),
                       [(scenes.PCON, scenes.Pcon((-30.0, -25.0, -20.0, 20.0, 25.0, 30.0), (0.0,) * 6,
                                                  (25.0, 25.0, 10.0, 10.0, 25.0, 25.0)), scenes._EYE, (0, 0, 0))])
    tr = tracks_from(np.array([[20.0, 0, 0], [40.0, 0, 0], [0.0, 0, 45.0]]), np.tile([1.0, 0, 0], (3, 1)))
    est, exact = orc.safety_estimate(sc, tr), orc.safety(sc, tr)
    assert est[0] == 0.0 and exact[0] == pytest.approx(10.0, rel=1e-15)
    assert est[1] == pytest.approx(15.0, rel=1e-15) and exact[1] == pytest.approx(math.sqrt(850.0), rel=1e-14)
    assert est[2] == pytest.approx(15.0, rel=1e-15) and exact[2] == pytest.approx(15.0, rel=1e-15)


def test_polycone_mother_inscribed_tube(orc):
    """pconm (outer radius 80 narrowing to 40 at z = 0, z -100..100, no
    daughter near the axis at z = +-90): its inscribed tube is r <= 40,
    |z| <= 100, so at (10, 0, 90) the mother's bound is min(40 - 10, 100 - 90)
    = 10, at (60, 0, 90), outside the tube, 0."""
    sc = scenes.Scene("m", scenes.PCON, scenes.pconm().mother_params, np.zeros(0, np.int32), np.zeros((0, 5)),
                      np.zeros((0, 9)), np.zeros((0, 3)), scenes.pconm().pdata)
    tr = tracks_from(np.array([[10.0, 0, 90.0], [60.0, 0, 90.0]]), np.tile([1.0, 0, 0], (2, 1)))
    est, exact = orc.safety_estimate(sc, tr), orc.safety(sc, tr)
    assert est[0] == 10.0 and exact[0] == 10.0
    assert est[1] == 0.0 and exact[1] == pytest.approx(10.0, rel=1e-15)


def test_cone_mother_inside_is_exact(orc):
    """Inside a cone mother (a convex meridian section) the least supporting
    line distance is the exact inside distance."""
    sc = scenes.Scene("cm", scenes.CONE, np.array([50.0, 10.0, 60.0, 20.0, 90.0]), np.zeros(0, np.int32),
                      np.zeros((0, 5)), np.zeros((0, 9)), np.zeros((0, 3)))
    rng = np.random.default_rng(5)
    p = rng.uniform(-90, 90, size=(20000, 3))
    tr = tracks_from(p, np.tile([1.0, 0, 0], (p.shape[0], 1)))
    inside = orc.contains(sc, tr) == -1
    est, exact = orc.safety_estimate(sc, tr), orc.safety(sc, tr)
    assert inside.mean() > 0.2
    assert np.allclose(est[inside], exact[inside], rtol=1e-13, atol=1e-12)
