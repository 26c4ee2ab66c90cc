"""Pins of the CPU oracle against facts fixed by geometry, not by the oracle.

* closed forms derived by hand (tests/golden/closed_forms.json)
* Cauchy's mean-chord theorem (4V/S for isotropic uniform random lines)
* invariants of the navigator (Fig. 1): the boundary point is where membership
  changes, safety <= step, the safety ball holds, exact symmetries of the scene
"""
import math

import numpy as np
import pytest

from helpers import expr, golden, scene_from_spec, tracks_from, points, dirs
from paper_1312_0816_gb300 import scenes


# ---------------------------------------------------------------- golden ---

@pytest.mark.parametrize("case", golden("closed_forms.json")["shape_cases"],
                         ids=lambda c: f"{c['q']}-k{c['kind']}-{c['x']}")
def test_shape_closed_form(orc, case):
    want = expr(case["expected"])
    if case["q"] in ("dist_out", "dist_in"):
        got, _ = orc.shape(case["kind"], case["p"], [case["x"]], [case["u"]], case["q"])
    else:
        got = orc.shape(case["kind"], case["p"], [case["x"]], None, case["q"])
    got = float(got[0])
    if math.isinf(want):
        assert math.isinf(got) and got > 0, case["why"]
    else:
        assert got == pytest.approx(want, rel=4e-16, abs=1e-13), case["why"]


@pytest.mark.parametrize("case", golden("closed_forms.json")["nav_cases"], ids=lambda c: c["why"][:40])
def test_navigator_closed_form(orc, case):
    sc = scene_from_spec(case["mother"], case["daughters"])
    r = orc.navigate(sc, tracks_from(case["p"], case["d"]))
    want = expr(case["step"])
    if math.isnan(want):
        assert math.isnan(r["step"][0])
    else:
        assert r["step"][0] == pytest.approx(want, rel=4e-16, abs=1e-13), case["why"]
    assert int(r["hit"][0]) == case["hit"], case["why"]


# ------------------------------------------------------------ mean chord ---

def _iur_chords(orc, kind, params, rb, n, seed):
    """Chords of isotropic uniform random lines through a ball of radius rb."""
    rng = np.random.default_rng(seed)
    u = np.stack(scenes.isotropic(rng, n), axis=1)
    a = np.where(np.abs(u[:, 0:1]) < 0.9, np.array([[1.0, 0, 0]]), np.array([[0, 1.0, 0]]))
    e1 = np.cross(u, a)
    e1 /= np.linalg.norm(e1, axis=1, keepdims=True)
    e2 = np.cross(u, e1)
    r = rb * np.sqrt(rng.uniform(size=(n, 1)))
    ph = rng.uniform(0, 2 * math.pi, size=(n, 1))
    w = r * (np.cos(ph) * e1 + np.sin(ph) * e2)
    L = 2.0 * rb
    s_in, _ = orc.shape(kind, params, w - L * u, u, "dist_out")
    s_back, _ = orc.shape(kind, params, w + L * u, -u, "dist_out")
    hit = np.isfinite(s_in)
    assert np.array_equal(hit, np.isfinite(s_back))
    return 2 * L - s_in[hit] - s_back[hit]


@pytest.mark.parametrize("kind,params,mean", [
    (0, (10.0, 20.0, 5.0), 4 * 10 * 20 * 5 / (10 * 20 + 20 * 5 + 5 * 10)),
    (1, (0.0, 15.0, 25.0), 4 * 15 * 25 / (2 * 25 + 15)),
    (2, (20.0, 0.0, 5.0, 0.0, 25.0), None),
    # solid wedge of 1 rad: V = dphi r^2 dz, S = dphi r^2 (caps) + dphi r 2dz + 2 r 2dz (phi faces)
    (3, (0.0, 10.0, 10.0, 0.0, 1.0), 4 * 1.0 * 100 * 10 / (1.0 * 100 + 1.0 * 10 * 20 + 2 * 10 * 20)),
])
def test_cauchy_mean_chord(orc, kind, params, mean):
    """Cauchy: E[chord] = 4V/S for IUR lines hitting a convex body."""
    if mean is None:  # solid frustum r1 -> r2 over height h
        h, r1, r2 = 2 * params[0], params[2], params[4]
        V = math.pi * h * (r1 * r1 + r1 * r2 + r2 * r2) / 3
        S = math.pi * (r1 + r2) * math.hypot(r2 - r1, h) + math.pi * (r1 * r1 + r2 * r2)
        mean = 4 * V / S
    rb = math.sqrt(sum(p * p for p in params)) + 1.0
    ch = _iur_chords(orc, kind, params, rb, 400_000, 11 + kind)
    se = ch.std() / math.sqrt(ch.size)
    assert abs(ch.mean() - mean) < 4 * se, (ch.mean(), mean, se)


# ------------------------------------------------------------ invariants ---

SCENES = [("box4", 0), ("toy40", 1), ("toy8", 1), ("diff3", None), ("seg4", None), ("pcon4", None),
          ("pconm", None)]


def _scene(name, seed):
    return scenes.SCENES[name]() if seed is None else scenes.SCENES[name](seed)


@pytest.mark.parametrize("name,seed", SCENES)
def test_boundary_point_membership_flips(orc, name, seed):
    """Just before the step the point is in the exclusive region (-1); just
    after it is inside the hit daughter, or outside the mother when the mother
    was hit."""
    sc = _scene(name, seed)
    tr = scenes.sample_tracks(sc, 3000, 21)
    r = orc.navigate(sc, tr)
    p, d = points(tr), dirs(tr)
    gap = r["second"] - r["step"]
    ok = gap > 1e-6
    before = tracks_from(p + (r["step"] - 1e-7)[:, None] * d, d)
    after = tracks_from(p + (r["step"] + 1e-7)[:, None] * d, d)
    wb = orc.contains(sc, before)
    wa = orc.contains(sc, after)
    assert np.all(wb[ok] == -1)
    expect_after = np.where(r["hit"] == -1, -2, r["hit"])
    # grazing hits may skim a corner and be outside again after 1e-7 mm
    frac = np.mean(wa[ok] == expect_after[ok])
    assert frac > 0.999, frac


@pytest.mark.parametrize("name,seed", SCENES)
def test_safety_bounds_step_and_ball(orc, name, seed):
    sc = _scene(name, seed)
    tr = scenes.sample_tracks(sc, 2000, 22)
    r = orc.navigate(sc, tr)
    saf = orc.safety(sc, tr)
    assert np.all(saf >= 0)
    assert np.all(saf <= r["step"] + 1e-9)
    # ball of radius 0.999*safety stays in the exclusive region
    rng = np.random.default_rng(5)
    p = points(tr)
    for _ in range(16):
        v = np.stack(scenes.isotropic(rng, tr.n), axis=1)
        q = p + 0.999 * saf[:, None] * v
        w = orc.contains(sc, tracks_from(q, v))
        assert np.all(w == -1)


def test_symmetry_box_mother_quarter_turn(orc):
    """A quarter turn about z maps the box mother onto itself exactly; turning
    daughters and tracks with it must leave steps and hits unchanged (up to
    the rounding of the re-ordered local-frame sums)."""
    sc = scenes.SCENES["diff3"]()
    tr = scenes.sample_tracks(sc, 4000, 23)
    Q = np.array([[0.0, -1.0, 0.0], [1.0, 0.0, 0.0], [0.0, 0.0, 1.0]])
    rot = np.array([(Q @ R.reshape(3, 3)).reshape(9) for R in sc.rot])
    sc2 = scenes.Scene("rot", sc.mother_kind, sc.mother_params, sc.kinds, sc.params, rot,
                       (Q @ sc.trans.T).T.copy())
    p2 = (Q @ points(tr).T).T
    d2 = (Q @ dirs(tr).T).T
    r1 = orc.navigate(sc, tr)
    r2 = orc.navigate(sc2, tracks_from(p2, d2))
    ok = (r1["second"] - r1["step"]) > 1e-9
    assert np.all(r1["hit"][ok] == r2["hit"][ok])
    assert np.allclose(r1["step"], r2["step"], rtol=0, atol=1e-9)


def test_symmetry_tube_mother_rotation(orc):
    sc = scenes.SCENES["toy40"](1)
    tr = scenes.sample_tracks(sc, 3000, 24)
    a = 0.73
    Q = np.array([[math.cos(a), -math.sin(a), 0.0], [math.sin(a), math.cos(a), 0.0], [0.0, 0.0, 1.0]])
    rot = np.array([(Q @ R.reshape(3, 3)).reshape(9) for R in sc.rot])
    sc2 = scenes.Scene("rot", sc.mother_kind, sc.mother_params, sc.kinds, sc.params, rot,
                       (Q @ sc.trans.T).T.copy())
    r1 = orc.navigate(sc, tr)
    r2 = orc.navigate(sc2, tracks_from((Q @ points(tr).T).T, (Q @ dirs(tr).T).T))
    ok = (r1["second"] - r1["step"]) > 1e-6
    assert np.all(r1["hit"][ok] == r2["hit"][ok])
    # rotation of inputs by an inexact matrix perturbs them by ~1e-13 mm
    assert np.max(np.abs(r1["step"] - r2["step"])[ok]) < 1e-8


def test_cone_equal_radii_is_tube(orc):
    """A cone whose radii do not change with z is a tube shell."""
    rng = np.random.default_rng(3)
    n = 20000
    x = rng.uniform(-60, 60, size=(n, 3))
    u = np.stack(scenes.isotropic(rng, n), axis=1)
    for q in ("dist_out", "dist_in"):
        a, _ = orc.shape(2, (25.0, 7.0, 30.0, 7.0, 30.0), x, u, q)
        b, _ = orc.shape(1, (7.0, 30.0, 25.0), x, u, q)
        fin = np.isfinite(b)
        assert np.array_equal(fin, np.isfinite(a))
        assert np.allclose(a[fin], b[fin], rtol=1e-15, atol=1e-12)


def test_box_slab_matches_axis_aligned_brute(orc):
    """Axis-aligned rays: the distance is a difference of coordinates."""
    rng = np.random.default_rng(4)
    h = np.array([7.0, 11.0, 13.0])
    n = 3000
    x = rng.uniform(-30, 30, size=(n, 3))
    ax = rng.integers(0, 3, size=n)
    sg = rng.choice([-1.0, 1.0], size=n)
    u = np.zeros((n, 3))
    u[np.arange(n), ax] = sg
    s, _ = orc.shape(0, tuple(h), x, u, "dist_out")
    for i in range(n):
        others = [k for k in range(3) if k != ax[i]]
        inside_others = all(abs(x[i, k]) <= h[k] for k in others)
        c = x[i, ax[i]] * sg[i]        # coordinate along the motion
        hh = h[ax[i]]
        if not inside_others or c > hh:
            want = math.inf
        elif c >= -hh:
            want = 0.0
        else:
            want = -hh - c
        assert s[i] == want


def test_tracks_are_in_exclusive_region(orc):
    for name, seed in SCENES:
        sc = _scene(name, seed)
        tr = scenes.sample_tracks(sc, 5000, 25)
        assert np.all(orc.contains(sc, tr) == -1)


def test_cone_hole_apex_on_end_face(orc):
    """A cone whose inner radius is 0 at z=-dz: its end face there is the full
    closed disk rho <= rmax1, so every line crossing that disk enters the solid
    at the plane, t = (-dz - z0)/uz, even when it then runs straight into the
    hole next to the apex (reading: closed solids; rho >= Rmin(z) holds where
    Rmin(z) = 0)."""
    rng = np.random.default_rng(12)
    p = (20.0, 0.0, 15.0, 5.0, 25.0)        # dz, rmin1=0, rmax1, rmin2, rmax2
    n = 20000
    rc = 10.0 ** rng.uniform(-12, -3, n)     # crossing radius: next to the apex
    ph = rng.uniform(0, 2 * math.pi, n)
    # steeper than the hole's slope 0.125, so the line enters the hole
    tilt = rng.uniform(0, 0.1, n)
    pa = rng.uniform(0, 2 * math.pi, n)
    u = np.stack([tilt * np.cos(pa), tilt * np.sin(pa), np.ones(n)], 1)
    cross = np.stack([rc * np.cos(ph), rc * np.sin(ph), np.full(n, -20.0)], 1)
    back = rng.uniform(1.0, 50.0, n)
    x = cross - back[:, None] * u
    want = (-20.0 - x[:, 2]) / u[:, 2]
    got, face = orc.shape(2, p, x, u, "dist_out")
    assert np.allclose(got, want, rtol=1e-14, atol=1e-12)
    # the on-axis line in closed form
    g, _ = orc.shape(2, p, [[0.0, 0.0, -100.0]], [[0.0, 0.0, 1.0]], "dist_out")
    assert g[0] == 80.0
