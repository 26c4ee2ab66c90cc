"""Pins of the oracle's polycone (kind 4: connected cone and tube sections,
Sec. 3.1; planes z[k] with radii rmin[k], rmax[k], cut to [sphi, sphi+dphi]).

Each pin is fixed by something other than the polycone code:
  - a polycone of two planes is the cone (kind 2) or, with equal radii, the
    tube and tube segment (kinds 1 and 3), pinned on their own;
  - a plane inserted on a section's radius lines changes nothing (the union
    of the two halves is the one section): the inner plane is no surface;
  - hand-derived closed forms on a non-convex bobbin;
  - Cauchy's mean chord 4V/S of a convex polycone with V and S in closed form;
  - the distances against a march along the ray with the membership test,
    which is the definition of the solid;
  - the safety against the nearest of many points sampled on the surface.
"""
import math

import numpy as np
import pytest

from paper_1312_0816_gb300 import scenes

Pcon = scenes.Pcon
TWO_PI = 2.0 * math.pi

# a solid bobbin: flanges of radius 25 (|z| in [25, 30]), slopes, a waist of radius 10
BOB = Pcon((-30.0, -25.0, -20.0, 20.0, 25.0, 30.0), (0.0,) * 6, (25.0, 25.0, 10.0, 10.0, 25.0, 25.0))
SHELL = Pcon((-25.0, -5.0, 5.0, 25.0), (5.0, 10.0, 10.0, 5.0), (15.0, 20.0, 20.0, 15.0))
WEDGE = Pcon((-20.0, 0.0, 20.0), (0.0, 5.0, 0.0), (20.0, 25.0, 15.0), -1.0, 4.2)
CONS = Pcon((-20.0, 20.0), (0.0, 5.0), (20.0, 10.0), 0.5, 1.3)
# limits and degenerate forms: pointed tips (outer radius 0 on the end
# planes), a pinch (the two sections meet in a circle at z = 0), the
# largest plane count
TIPS = Pcon((-20.0, 0.0, 20.0), (0.0, 0.0, 0.0), (0.0, 15.0, 0.0))
PINCH = Pcon((-20.0, 0.0, 20.0), (5.0, 10.0, 5.0), (15.0, 10.0, 15.0), 0.3, 5.0)
ZIG32 = Pcon(tuple(-31.0 + 2.0 * k for k in range(32)), tuple(1.0 + (k % 3) for k in range(32)),
             tuple(6.0 + 4.0 * (k % 2) + 0.2 * k for k in range(32)))
ALL = [BOB, SHELL, WEDGE, CONS, TIPS, PINCH, ZIG32]
IDS = ["bobbin", "shell", "wedge", "cons", "tips", "pinch", "zig32"]


def rays(n, seed, box=60.0):
    rng = np.random.default_rng(seed)
    x = rng.uniform(-box, box, size=(n, 3))
    u = np.stack(scenes.isotropic(rng, n), axis=1)
    return x, u


def sec_face(f, outer=6, inner=7):
    """Section faces 16 + 2k (outer) / 17 + 2k (inner) -> the cone's 6 / 7."""
    f = f.copy()
    sec = f >= 16
    f[sec] = np.where((f[sec] - 16) % 2 == 0, outer, inner)
    return f


# ----------------------------------------------------- reductions to kinds 1-3

@pytest.mark.parametrize("seed", range(4))
def test_two_planes_is_the_cone(orc, seed):
    rng = np.random.default_rng(100 + seed)
    dz = rng.uniform(5.0, 30.0)
    r1, r2 = rng.uniform(5.0, 30.0, size=2)
    i1, i2 = rng.uniform(0.0, 0.8) * r1, rng.uniform(0.0, 0.8) * r2
    if seed == 0:
        i1 = 0.0          # an inner apex on the -z plane
    pc = Pcon((-dz, dz), (i1, i2), (r1, r2))
    cone = (dz, i1, r1, i2, r2)
    x, u = rays(20000, seed, 1.5 * max(dz, r1, r2))
    for what in ("dist_out", "dist_in"):
        a, fa = orc.shape(scenes.PCON, pc, x, u, what)
        b, fb = orc.shape(scenes.CONE, cone, x, u, what)
        assert np.array_equal(np.isinf(a), np.isinf(b))
        fin = np.isfinite(b)
        assert np.allclose(a[fin], b[fin], rtol=1e-14, atol=1e-13)
        assert np.mean(sec_face(fa) == fb) > 0.9999
    assert np.array_equal(orc.shape(scenes.PCON, pc, x, None, "contains"),
                          orc.shape(scenes.CONE, cone, x, None, "contains"))
    for what in ("safety_out", "safety_in"):
        assert np.allclose(orc.shape(scenes.PCON, pc, x, None, what), orc.shape(scenes.CONE, cone, x, None, what),
                           rtol=1e-14, atol=1e-13)


@pytest.mark.parametrize("sphi,dphi", [(0.0, TWO_PI), (0.3, 1.2), (2.0, math.pi), (-1.0, 4.5)])
def test_equal_radii_is_the_tube_segment(orc, sphi, dphi):
    pc = Pcon((-15.0, 15.0), (5.0, 5.0), (25.0, 25.0), sphi, dphi)
    tubs = (5.0, 25.0, 15.0, sphi, dphi)
    x, u = rays(20000, 7, 40.0)
    for what in ("dist_out", "dist_in"):
        a, fa = orc.shape(scenes.PCON, pc, x, u, what)
        b, fb = orc.shape(scenes.TUBS, tubs, x, u, what)
        assert np.array_equal(np.isinf(a), np.isinf(b))
        fin = np.isfinite(b)
        assert np.allclose(a[fin], b[fin], rtol=1e-14, atol=1e-13)
        assert np.mean(sec_face(fa) == fb) > 0.9999
    assert np.array_equal(orc.shape(scenes.PCON, pc, x, None, "contains"),
                          orc.shape(scenes.TUBS, tubs, x, None, "contains"))
    for what in ("safety_out", "safety_in"):
        assert np.allclose(orc.shape(scenes.PCON, pc, x, None, what), orc.shape(scenes.TUBS, tubs, x, None, what),
                           rtol=1e-14, atol=1e-13)


@pytest.mark.parametrize("dphi", [TWO_PI, 1.1, 4.0])
def test_plane_on_the_radius_lines_is_no_surface(orc, dphi):
    """Radii (2, 4, 6) and (10, 15, 20) at z = (-20, 0, 20) lie on straight
    lines, so the two sections are the one cone (20, 2, 10, 6, 20): a track
    crossing z = 0 inside does not stop there."""
    three = Pcon((-20.0, 0.0, 20.0), (2.0, 4.0, 6.0), (10.0, 15.0, 20.0), 0.4, dphi)
    two = Pcon((-20.0, 20.0), (2.0, 6.0), (10.0, 20.0), 0.4, dphi)
    x, u = rays(20000, 8, 30.0)
    for what in ("dist_out", "dist_in"):
        a, fa = orc.shape(scenes.PCON, three, x, u, what)
        b, fb = orc.shape(scenes.PCON, two, x, u, what)
        fin = np.isfinite(b)
        assert np.array_equal(np.isinf(a), np.isinf(b))
        assert np.allclose(a[fin], b[fin], rtol=1e-13, atol=1e-12)
        assert np.mean(sec_face(fa) == sec_face(fb)) > 0.9999
        assert not np.any(fa[fin & (a > 0)] == -1)   # never an inner plane
    for what in ("safety_out", "safety_in"):
        assert np.allclose(orc.shape(scenes.PCON, three, x, None, what),
                           orc.shape(scenes.PCON, two, x, None, what), rtol=1e-13, atol=1e-12)


# ------------------------------------------------------------- closed forms

def one(orc, pc, x, u, what):
    out = orc.shape(scenes.PCON, pc, [x], [u] if u is not None else None, what)
    if isinstance(out, tuple):
        return float(out[0][0]), int(out[1][0])
    return float(out[0])


@pytest.mark.parametrize("x,u,want,face", [
    ((50.0, 0.0, 0.0), (-1.0, 0.0, 0.0), 40.0, 20),            # the waist (section 2)
    ((50.0, 0.0, 27.0), (-1.0, 0.0, 0.0), 25.0, 24),           # a flange (section 4)
    # r = 20 on the slope of section 3 (10 -> 25 over z 20 -> 25): z = 20 + 10/3
    ((20.0, 0.0, 0.0), (0.0, 0.0, 1.0), 20.0 + 10.0 / 3.0, 22),
    ((5.0, 0.0, -40.0), (0.0, 0.0, 1.0), 10.0, 4),             # the -z end plane
    ((30.0, 0.0, 0.0), (0.0, 0.0, 1.0), math.inf, -1),          # beside it
])
def test_bobbin_dist_out(orc, x, u, want, face):
    s, f = one(orc, BOB, x, u, "dist_out")
    assert (s == pytest.approx(want, rel=1e-14, abs=1e-13)) if math.isfinite(want) else math.isinf(s)
    assert f == face


@pytest.mark.parametrize("x,u,want,face", [
    ((0.0, 0.0, 0.0), (1.0, 0.0, 0.0), 10.0, 20),
    ((0.0, 0.0, 0.0), (0.0, 0.0, 1.0), 30.0, 5),              # crosses four inner planes
    # from the flange down across z = 25 into the slope: r = 15 at z = 20 + 5/3
    ((15.0, 0.0, 27.0), (0.0, 0.0, -1.0), 27.0 - (20.0 + 5.0 / 3.0), 22),
])
def test_bobbin_dist_in(orc, x, u, want, face):
    s, f = one(orc, BOB, x, u, "dist_in")
    assert s == pytest.approx(want, rel=1e-14, abs=1e-13)
    assert f == face


def test_bobbin_contains_and_safety(orc):
    assert one(orc, BOB, (9.0, 0.0, 0.0), None, "contains") == 1.0
    assert one(orc, BOB, (11.0, 0.0, 0.0), None, "contains") == 0.0
    assert one(orc, BOB, (24.0, 0.0, 27.0), None, "contains") == 1.0
    assert one(orc, BOB, (0.0, 0.0, 0.0), None, "safety_in") == pytest.approx(10.0, abs=1e-14)
    assert one(orc, BOB, (0.0, 0.0, 29.0), None, "safety_in") == pytest.approx(1.0, abs=1e-14)
    # nearest point of the section (r, z) = (25, 25): the flange's inner rim
    assert one(orc, BOB, (50.0, 0.0, 0.0), None, "safety_out") == pytest.approx(25.0 * math.sqrt(2.0), rel=1e-15)
    assert one(orc, BOB, (0.0, 30.0, 0.0), None, "safety_out") == pytest.approx(20.0, rel=1e-15)


def test_wedge_closed_form(orc):
    """WEDGE: azimuths [-1, 3.2]; the excluded sector is around phi = 4.2."""
    ex = (10.0 * math.cos(4.2), 10.0 * math.sin(4.2), 0.0)
    assert one(orc, WEDGE, ex, None, "contains") == 0.0
    assert one(orc, WEDGE, (10.0, 0.0, 0.0), None, "contains") == 1.0
    # inside at phi = 0, r = 10, z = 0: the inner radius is 5 there, so the
    # hole is 5 away; the faces at -1 and 3.2 rad are 10 sin(1) = 8.41 away
    assert one(orc, WEDGE, (10.0, 0.0, 0.0), None, "safety_in") == pytest.approx(5.0, abs=1e-14)
    # through the axis at z = 0 the track meets the hole (radius 5) and enters
    # through the inner surface on the far side
    s, f = one(orc, WEDGE, (20.0 * math.cos(4.2), 20.0 * math.sin(4.2), 0.0),
               (-math.cos(4.2), -math.sin(4.2), 0.0), "dist_out")
    assert s == pytest.approx(25.0, rel=1e-14) and f in (17, 19)
    # tangentially from r = 10 at phi = 4.2 the azimuth grows as 4.2 + atan(s/10)
    # and reaches the face at sphi = -1 (= 2 pi - 1) at r = 21.3 (in [5, 25])
    s, f = one(orc, WEDGE, (10.0 * math.cos(4.2), 10.0 * math.sin(4.2), 0.0),
               (-math.sin(4.2), math.cos(4.2), 0.0), "dist_out")
    assert s == pytest.approx(10.0 * math.tan(2.0 * math.pi - 5.2), rel=1e-13) and f == 8


# ---------------------------------------------------------------- mean chord

def test_cauchy_mean_chord_convex_polycone(orc):
    """A convex polycone (solid double frustum 10 -> 20 -> 10 over z -20..20,
    cut to a 1.2 rad wedge): E[chord] = 4V/S for isotropic uniform random
    lines, V and S of the wedge in closed form."""
    from test_oracle_pins import _iur_chords

    dphi = 1.2
    pc = Pcon((-20.0, 0.0, 20.0), (0.0, 0.0, 0.0), (10.0, 20.0, 10.0), 0.0, dphi)
    h, r1, r2 = 20.0, 10.0, 20.0
    frac = dphi / TWO_PI
    V = 2 * frac * math.pi * h * (r1 * r1 + r1 * r2 + r2 * r2) / 3
    lateral = 2 * frac * math.pi * (r1 + r2) * math.hypot(r2 - r1, h)
    caps = 2 * frac * math.pi * r1 * r1
    faces = 2 * (2 * h * (r1 + r2) / 2)             # two trapezoids of the cross-section
    mean = 4 * V / (lateral + caps + faces)
    ch = _iur_chords(orc, scenes.PCON, pc, 31.0, 400_000, 19)
    se = ch.std() / math.sqrt(ch.size)
    assert abs(ch.mean() - mean) < 4 * se, (ch.mean(), mean, se)


# ------------------------------------------------- against the membership test

@pytest.mark.parametrize("pc", ALL, ids=IDS)
def test_distances_against_membership_march(orc, pc):
    """Before DistFromOutside every point of the ray is outside, just after it
    inside; before DistFromInside every point is inside, just after it
    outside (sampled every 0.05 mm; rays grazing within 1e-6 mm excepted)."""
    x, u = rays(600, 11, 40.0)
    so, _ = orc.shape(scenes.PCON, pc, x, u, "dist_out")
    si, _ = orc.shape(scenes.PCON, pc, x, u, "dist_in")
    inside = orc.shape(scenes.PCON, pc, x, None, "contains") == 1.0
    eps = 1e-6
    checked = 0
    for i in range(x.shape[0]):
        if inside[i]:
            assert so[i] == 0.0
            end = si[i]
            t = np.arange(0.0, max(end - eps, 0.0), 0.05)
            pts = x[i] + t[:, None] * u[i]
            assert np.all(orc.shape(scenes.PCON, pc, pts, None, "contains") == 1.0), i
            after = orc.shape(scenes.PCON, pc, [x[i] + (end + eps) * u[i]], None, "contains")[0]
            checked += after == 0.0
        elif np.isfinite(so[i]):
            t = np.arange(0.0, so[i] - eps, 0.05)
            pts = x[i] + t[:, None] * u[i]
            assert np.all(orc.shape(scenes.PCON, pc, pts, None, "contains") == 0.0), i
            after = orc.shape(scenes.PCON, pc, [x[i] + (so[i] + eps) * u[i]], None, "contains")[0]
            checked += after == 1.0
        else:
            t = np.arange(0.0, 200.0, 0.05)
            pts = x[i] + t[:, None] * u[i]
            assert np.all(orc.shape(scenes.PCON, pc, pts, None, "contains") == 0.0), i
            checked += 1
    assert checked >= 0.995 * x.shape[0]


def surface_points(pc, n, seed):
    """Points on the polycone's surface: caps, section surfaces, phi faces."""
    rng = np.random.default_rng(seed)
    z, rn, rx = (np.asarray(a, float) for a in (pc.z, pc.rmin, pc.rmax))
    out = []
    m = n // 4
    for kind in range(4):
        ph = pc.sphi + pc.dphi * rng.uniform(size=m)
        if kind == 0:                                  # end caps
            top = rng.uniform(size=m) < 0.5
            zz = np.where(top, z[-1], z[0])
            lo, hi = np.where(top, rn[-1], rn[0]), np.where(top, rx[-1], rx[0])
            r = lo + (hi - lo) * rng.uniform(size=m)
        elif kind in (1, 2):                           # outer / inner section surfaces
            rr = rx if kind == 1 else rn
            real = np.nonzero(rr[:-1] + rr[1:] > 0)[0]   # an inner radius 0 at both ends is the axis
            if real.size == 0:
                continue
            k = real[rng.integers(0, real.size, size=m)]
            f = rng.uniform(size=m)
            r = rr[k] + (rr[k + 1] - rr[k]) * f
            zz = z[k] + (z[k + 1] - z[k]) * f
        else:                                          # phi faces
            if pc.dphi >= TWO_PI:
                continue
            ph = pc.sphi + pc.dphi * (rng.uniform(size=m) < 0.5)
            k = rng.integers(0, len(z) - 1, size=m)
            f = rng.uniform(size=m)
            zz = z[k] + (z[k + 1] - z[k]) * f
            lo = rn[k] + (rn[k + 1] - rn[k]) * f
            hi = rx[k] + (rx[k + 1] - rx[k]) * f
            r = lo + (hi - lo) * rng.uniform(size=m)
        out.append(np.stack([r * np.cos(ph), r * np.sin(ph), zz], axis=1))
    return np.concatenate(out)


@pytest.mark.parametrize("pc", ALL, ids=IDS)
def test_safety_against_sampled_surface(orc, pc):
    """Exact safety <= distance to every surface point, and within the
    sampling resolution of the nearest sampled one."""
    surf = surface_points(pc, 400_000, 3)
    x, _ = rays(300, 12, 40.0)
    inside = orc.shape(scenes.PCON, pc, x, None, "contains") == 1.0
    sin_ = orc.shape(scenes.PCON, pc, x, None, "safety_in")
    sout = orc.shape(scenes.PCON, pc, x, None, "safety_out")
    saf = np.where(inside, sin_, sout)
    for i in range(x.shape[0]):
        d = np.sqrt(((surf - x[i]) ** 2).sum(axis=1)).min()
        assert saf[i] <= d + 1e-9, i
        assert saf[i] >= d - 0.6, (i, saf[i], d)
