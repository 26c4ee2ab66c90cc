"""Brute-force pins of the oracle on small inputs.

* Ray marching with the oracle's own membership test (Contains) and 60
  bisection steps finds where a track leaves the exclusive region of the mother;
  that must be the navigator's step (Fig. 1) up to the marching's blind spot
  (chords shorter than the march step).
* Sphere tracing with the exact safety never overshoots a boundary, so it
  converges to the same step.
* The exact safety is the distance to the nearest boundary point: the minimum
  of the step over many directions approaches it from above.
"""
import math

import numpy as np
import pytest

from helpers import points, dirs, tracks_from
from paper_1312_0816_gb300 import scenes


def _march(orc, sc, tr, h, smax):
    p, d = points(tr), dirs(tr)
    n = tr.n
    s = np.zeros(n)
    done = np.zeros(n, dtype=bool)
    lo = np.zeros(n)
    hi = np.full(n, np.nan)
    while not done.all():
        idx = np.nonzero(~done)[0]
        s_next = s[idx] + h
        q = p[idx] + s_next[:, None] * d[idx]
        w = orc.contains(sc, tracks_from(q, d[idx]))
        left = w != -1
        hi[idx[left]] = s_next[left]
        lo[idx[left]] = s[idx[left]]
        done[idx[left]] = True
        s[idx] = s_next
        done[idx[s_next > smax]] = True
    for _ in range(60):
        mid = 0.5 * (lo + hi)
        w = orc.contains(sc, tracks_from(p + mid[:, None] * d, d))
        inside = w == -1
        lo = np.where(inside, mid, lo)
        hi = np.where(inside, hi, mid)
    return hi


def _extent(sc):
    """Largest coordinate of the mother."""
    if sc.mother_kind == scenes.PCON:
        z, _, rx = sc.planes_of(sc.mother_params)
        return float(max(np.abs(z).max(), rx.max()))
    return float(np.max(sc.mother_params))


@pytest.mark.parametrize("name,seed,n,h", [("box4", 0, 10000, 1.25), ("diff3", None, 10000, 0.6),
                                           ("seg4", None, 6000, 0.6), ("pcon4", None, 6000, 0.6),
                                           ("pconm", None, 6000, 0.6), ("toy8", 1, 1500, 3.5)])
def test_ray_marching_agrees(orc, name, seed, n, h):
    sc = scenes.SCENES[name]() if seed is None else scenes.SCENES[name](seed)
    tr = scenes.sample_tracks(sc, n, 31)
    r = orc.navigate(sc, tr, nthreads=4)
    smax = 2.0 * _extent(sc) * 1.8
    sm = _march(orc, sc, tr, h, smax)
    # marching finds the first membership change at march resolution, so it
    # can only be later than the true step (it may jump over a short chord)
    diff = sm - r["step"]
    assert np.all(diff > -1e-9), diff.min()
    agree = np.abs(diff) <= 1e-9
    assert agree.mean() > 0.995, agree.mean()
    # every disagreement is a skipped chord: the track re-enters the exclusive
    # region within one march step after the oracle's boundary point (a chord
    # of a daughter; or, in a mother that is not convex, of the outside)
    bad = np.nonzero(~agree)[0]
    if bad.size:
        p, d = points(tr)[bad], dirs(tr)[bad]
        sub = tracks_from(p, d)
        rs = orc.navigate(sc, sub)
        assert np.all(rs["hit"] >= (-1 if sc.mother_kind == scenes.PCON else 0))
        q = p + (r["step"][bad] + h)[:, None] * d
        w = orc.contains(sc, tracks_from(q, d))
        assert np.all(w == -1)


@pytest.mark.parametrize("name,seed", [("box4", 0), ("diff3", None), ("toy40", 1), ("seg4", None),
                                       ("pcon4", None), ("pconm", None)])
def test_sphere_tracing_agrees(orc, name, seed):
    sc = scenes.SCENES[name]() if seed is None else scenes.SCENES[name](seed)
    tr = scenes.sample_tracks(sc, 3000, 32)
    r = orc.navigate(sc, tr, nthreads=4)
    p, d = points(tr), dirs(tr)
    s = np.zeros(tr.n)
    for _ in range(4000):
        saf = orc.safety(sc, tracks_from(p + s[:, None] * d, d), nthreads=4)
        s = s + saf
    conv = orc.safety(sc, tracks_from(p + s[:, None] * d, d)) < 1e-11
    # never overshoots
    assert np.all(s <= r["step"] + 1e-9)
    assert conv.mean() > 0.97, conv.mean()
    assert np.max(np.abs(s - r["step"])[conv]) < 1e-9


@pytest.mark.parametrize("name,seed", [("diff3", None), ("toy8", 1), ("seg4", None), ("pcon4", None),
                                       ("pconm", None)])
def test_safety_is_exact_distance(orc, name, seed):
    """min over 20000 directions of the step >= safety and within the angular
    resolution of it (an under-estimating safety would fail the upper side)."""
    sc = scenes.SCENES[name]() if seed is None else scenes.SCENES[name](seed)
    tr = scenes.sample_tracks(sc, 40, 33)
    saf = orc.safety(sc, tr)
    m = 20000
    k = np.arange(m) + 0.5
    th = np.arccos(1 - 2 * k / m)
    ph = math.pi * (1 + 5 ** 0.5) * k
    v = np.stack([np.cos(ph) * np.sin(th), np.sin(ph) * np.sin(th), np.cos(th)], axis=1)
    spacing = math.sqrt(4 * math.pi / m)
    for i in range(tr.n):
        p0 = points(tr)[i:i + 1]
        r = orc.navigate(sc, tracks_from(np.repeat(p0, m, axis=0), v), nthreads=4)
        assert r["step"].min() >= saf[i] - 1e-9
        # refine around the 4 best directions on ever finer local grids; near
        # an edge or corner the step grows linearly with the angular error
        cand = v[np.argsort(r["step"])[:4]]
        best = r["step"].min()
        for c in cand:
            width = 2 * spacing
            for _ in range(4):
                a = np.where(abs(c[0]) < 0.9, np.array([1.0, 0, 0]), np.array([0, 1.0, 0]))
                e1 = np.cross(c, a)
                e1 /= np.linalg.norm(e1)
                e2 = np.cross(c, e1)
                g = np.linspace(-width, width, 21)
                gu, gv = np.meshgrid(g, g)
                w = c[None, :] + gu.reshape(-1, 1) * e1 + gv.reshape(-1, 1) * e2
                w /= np.linalg.norm(w, axis=1, keepdims=True)
                rr = orc.navigate(sc, tracks_from(np.repeat(p0, w.shape[0], axis=0), w))
                k = int(np.argmin(rr["step"]))
                assert rr["step"][k] >= saf[i] - 1e-9
                c = w[k]
                best = min(best, rr["step"][k])
                width /= 8
        assert best <= saf[i] * (1 + 1e-4) + 1e-9, (i, best, saf[i])
