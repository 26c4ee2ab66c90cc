"""Per-shape queries (Sec. 3.1, measured per shape in Fig. 2) on the GPU
against the oracle's shape routines: DistFromOutside, DistFromInside, the two
safeties and Contains of one Box, Tube, Cone, tube segment or polycone, in
its own frame and placed.

Bars: every distance within max(1e-9 mm, err) of the oracle's, err the
oracle's a-priori FP64 error bound of that query (pinned against exact
crossings in test_oracle_errbound.py), and the crossed face equal unless
another of the solid's surfaces is crossed within that tolerance (an edge, a
rim); a point within 1e-9 mm of the surface is inside or outside by rounding,
so its distances are not unique and only counted.  Where the two answers
differ by more, the GPU's must be the oracle's for the start point moved by
1e-9 mm along some axis (a ray grazing a cylinder or cone: FP64 rounding
decides between touch and miss); those are counted and capped.  Safeties within 1e-9 mm; Contains exact outside the
1e-9 mm surface band.
"""
import math

import numpy as np
import pytest

from helpers import PERTURB, PERTURB_MATCH
from paper_1312_0816_gb300 import scenes

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-9

SOLIDS = [
    (0, (10.0, 20.0, 30.0)),
    (1, (0.0, 20.0, 30.0)),
    (1, (5.0, 20.0, 30.0)),
    (2, (30.0, 0.0, 10.0, 0.0, 20.0)),
    (2, (30.0, 5.0, 10.0, 8.0, 20.0)),
    (2, (30.0, 0.0, 10.0, 5.0, 20.0)),
    (2, (30.0, 0.0, 0.0, 0.0, 20.0)),
    (3, (0.0, 10.0, 10.0, 0.0, math.pi / 2)),         # tube segments: a solid quarter,
    (3, (4.0, 10.0, 10.0, 0.5, 1.5 * math.pi)),       # a non-convex shell wedge,
    (3, (2.0, 10.0, 8.0, -1.0, math.pi)),             # a half shell (both faces in one plane),
    (3, (0.0, 10.0, 8.0, 2.0, 0.2)),                  # a thin wedge,
    (3, (3.0, 10.0, 8.0, 0.3, 2 * math.pi)),          # a whole turn
    # polycones: a solid bobbin (not convex), a shell whose hole widens, a
    # non-convex wedge with inner apexes on its end planes, a cone segment, a
    # hollow cone segment beyond a half turn, and a zigzag of 12 planes
    (4, scenes.Pcon((-30.0, -25.0, -20.0, 20.0, 25.0, 30.0), (0.0,) * 6, (25.0, 25.0, 10.0, 10.0, 25.0, 25.0))),
    (4, scenes.Pcon((-25.0, -5.0, 5.0, 25.0), (5.0, 10.0, 10.0, 5.0), (15.0, 20.0, 20.0, 15.0))),
    (4, scenes.Pcon((-20.0, 0.0, 20.0), (0.0, 5.0, 0.0), (20.0, 25.0, 15.0), -1.0, 4.2)),
    (4, scenes.Pcon((-20.0, 20.0), (0.0, 5.0), (20.0, 10.0), 0.5, 1.3)),
    (4, scenes.Pcon((-15.0, 15.0), (4.0, 8.0), (12.0, 18.0), 2.0, 3.9)),
    (4, scenes.Pcon(tuple(-33.0 + 6.0 * k for k in range(12)), tuple(2.0 + (k % 2) * 3.0 for k in range(12)),
                    tuple(10.0 + (k % 2) * 8.0 + k for k in range(12)))),
    # limits: pointed tips, a pinch in a non-convex wedge, the largest plane count
    (4, scenes.Pcon((-20.0, 0.0, 20.0), (0.0, 0.0, 0.0), (0.0, 15.0, 0.0))),
    (4, scenes.Pcon((-20.0, 0.0, 20.0), (5.0, 10.0, 5.0), (15.0, 10.0, 15.0), 0.3, 5.0)),
    (4, scenes.Pcon(tuple(-31.0 + 2.0 * k for k in range(32)), tuple(1.0 + (k % 3) for k in range(32)),
                    tuple(6.0 + 4.0 * (k % 2) + 0.2 * k for k in range(32)))),
]
WHAT = {"dist_out": 0, "dist_in": 1, "safety_out": 2, "safety_in": 3, "contains": 4}


@pytest.fixture(scope="module")
def g():
    import paper_1312_0816_gb300 as pkg

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    pkg.load()
    return pkg


def extent(kind, p):
    if kind == 0:
        return np.array(p[:3])
    if kind == 4:
        r = max(p.rmax)
        return np.array([r, r, max(abs(p.z[0]), abs(p.z[-1]))])
    if kind in (1, 3):
        return np.array([p[1], p[1], p[2]])
    r = max(p[2], p[4])
    return np.array([r, r, p[0]])


def sample(kind, p, n, seed):
    rng = np.random.default_rng(seed)
    x = rng.uniform(-1.5, 1.5, size=(n, 3)) * extent(kind, p)
    u = np.stack(scenes.isotropic(rng, n), axis=1)
    return x, u


def on_surface(orc, kind, p, x, u):
    """Points on the surface: the oracle's DistFromOutside hits, moved by
    0, +-1e-12 and +-1e-7 mm along the ray."""
    s, _ = orc.shape(kind, p, x, u, "dist_out")
    m = np.isfinite(s) & (s > 0)
    hit = x[m] + s[m, None] * u[m]
    pts = [hit + e * u[m] for e in (0.0, 1e-12, -1e-12, 1e-7, -1e-7)]
    dirs = [u[m]] * 5
    return np.concatenate(pts), np.concatenate(dirs)


def gpu(g, kind, p, what, x, u, rot=None, trans=None):
    t = [torch.from_numpy(np.ascontiguousarray(x[:, k])).cuda() for k in range(3)]
    d = [torch.from_numpy(np.ascontiguousarray(u[:, k])).cuda() for k in range(3)]
    out, face = g.geo_shape_query(kind, p, WHAT[what], *t, *d, rot=rot, trans=trans, want_face=True)
    torch.cuda.synchronize()
    return out.cpu().numpy(), face.cpu().numpy()


def check_distance(orc, kind, p, what, x, u, got, gface, tnorm=0.0):
    """Every ray checked; returns the number decided by rounding."""
    want, wface = orc.shape(kind, p, x, u, what)
    err, gap = orc.shape_err(kind, p, x, u, what, tnorm)
    tol = np.maximum(TOL, err)
    both_inf = np.isinf(got) & np.isinf(want)
    with np.errstate(invalid="ignore"):
        close = both_inf | (np.abs(got - want) <= tol)
    far = np.nonzero(~close)[0]
    if far.size:
        # a grazing contact decided by rounding: the GPU's answer is the
        # oracle's for the start point moved by 1e-9 mm along some axis
        ok = np.zeros(far.size, dtype=bool)
        for k in range(3):
            for sg in (-1.0, 1.0):
                xm = x[far].copy()
                xm[:, k] += sg * PERTURB
                wm, _ = orc.shape(kind, p, xm, u[far], what)
                em, _ = orc.shape_err(kind, p, xm, u[far], what, tnorm)
                with np.errstate(invalid="ignore"):
                    ok |= (np.isinf(wm) & np.isinf(got[far])) | (np.abs(got[far] - wm) <= np.maximum(PERTURB_MATCH, em))
        assert np.all(ok), (far[~ok][:5], got[far][~ok][:5], want[far][~ok][:5])
    free = ~close | both_inf | (want <= tol) | (gap <= tol)
    fbad = np.nonzero(~free & (gface != wface))[0]
    assert fbad.size == 0, (fbad[:5], gface[fbad][:5], wface[fbad][:5], got[fbad][:5], want[fbad][:5])
    return int(far.size)


@pytest.mark.parametrize("idx", range(len(SOLIDS)))
def test_shape_queries_match_oracle(g, orc, idx):
    kind, p = SOLIDS[idx]
    x, u = sample(kind, p, 200000, 100 + idx)
    xs, us = on_surface(orc, kind, p, x[:20000], u[:20000])
    for pts, dirs, max_touch in ((x, u, 1e-5), (xs, us, 2e-3)):
        # within 1e-9 mm of the surface, inside/outside (and so both
        # distances) is decided by rounding: that band is only counted
        band = orc.shape(kind, p, pts, None, "safety_out") + orc.shape(kind, p, pts, None, "safety_in") < TOL
        for what in ("dist_out", "dist_in"):
            got, gface = gpu(g, kind, p, what, pts, dirs)
            touch = check_distance(orc, kind, p, what, pts[~band], dirs[~band], got[~band], gface[~band])
            assert touch <= max_touch * pts.shape[0], touch
        for what in ("safety_out", "safety_in"):
            got, gface = gpu(g, kind, p, what, pts, dirs)
            want = orc.shape(kind, p, pts, None, what)
            assert np.max(np.abs(got - want)) <= TOL, what
            assert np.all(gface == -1)
        got, _ = gpu(g, kind, p, "contains", pts, dirs)
        want = orc.shape(kind, p, pts, None, "contains")
        assert np.array_equal(got[~band], want[~band])


@pytest.mark.parametrize("idx", [0, 2, 4, 8, 12, 14])
def test_placed_solid(g, orc, idx):
    """Placement applied in the kernel: compare with the oracle on points
    transformed on the host (the transforms round differently: the error
    bound counts the placement's distance)."""
    kind, p = SOLIDS[idx]
    rng = np.random.default_rng(7 + idx)
    R = np.asarray(scenes.haar_rotation(rng)).reshape(3, 3)
    t = np.array([120.0, -40.0, 75.0])
    xl, ul = sample(kind, p, 50000, 200 + idx)
    xw = xl @ R.T + t
    uw = ul @ R.T
    x_back = (xw - t) @ R
    u_back = uw @ R
    for what in ("dist_out", "dist_in"):
        got, gface = gpu(g, kind, p, what, xw, uw, rot=R, trans=t)
        touch = check_distance(orc, kind, p, what, x_back, u_back, got, gface, tnorm=float(np.linalg.norm(t)))
        assert touch <= 1e-4 * xw.shape[0], touch
    got, _ = gpu(g, kind, p, "safety_out", xw, uw, rot=R, trans=t)
    want = orc.shape(kind, p, x_back, None, "safety_out")
    assert np.max(np.abs(got - want)) <= 1e-9 * 300


def test_invalid_inputs(g):
    x = np.array([[np.nan, 0, 0], [0, np.inf, 0], [1.0, 2.0, 3.0]])
    u = np.array([[1.0, 0, 0], [1.0, 0, 0], [0.0, 0.0, 0.0]])
    for what in ("dist_out", "dist_in"):
        got, face = gpu(g, 1, (5.0, 20.0, 30.0), what, x, u)
        assert np.all(np.isnan(got)) and np.all(face == -1)
    got, _ = gpu(g, 1, (5.0, 20.0, 30.0), "safety_out", x[:2], u[:2])
    assert np.all(np.isnan(got))
