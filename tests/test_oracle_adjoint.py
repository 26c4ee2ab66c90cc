"""Pins of the oracle's adjoint (gradient of the navigator step).

The adjoint follows the implicit-function rule on the winning surface; it is
pinned by central finite differences of the oracle's own step (an independent
route to the same derivative) and by exact values for axis-aligned faces.
"""
import numpy as np
import pytest

from helpers import points, dirs, tracks_from
from paper_1312_0816_gb300 import scenes

H = 1e-6


def _smooth_mask(orc, sc, tr, r):
    """Tracks whose (winner, face) is unchanged under +-1e-3 mm moves of the
    start point and whose tie gap exceeds 1e-3 mm."""
    ok = (r["second"] - r["step"]) > 1e-3
    ok &= r["hit"] >= -1
    p, d = points(tr), dirs(tr)
    for k in range(3):
        for sg in (-1.0, 1.0):
            q = p.copy()
            q[:, k] += sg * 1e-3
            rr = orc.navigate(sc, tracks_from(q, d))
            ok &= (rr["hit"] == r["hit"]) & (rr["face"] == r["face"])
    return ok


def _fd_tracks(orc, sc, tr, which, k, h=H):
    p, d = points(tr), dirs(tr)
    a, b = (p.copy(), d.copy()), (p.copy(), d.copy())
    idx = 0 if which == "p" else 1
    a[idx][:, k] += h
    b[idx][:, k] -= h
    sa = orc.navigate(sc, tracks_from(*a))["step"]
    sb = orc.navigate(sc, tracks_from(*b))["step"]
    return (sa - sb) / (2 * h)


def _truncation(orc, sc, tr, which, k, fd):
    """Truncation error of the central difference, estimated from a second
    quotient at h/2 (4/3 of their difference); large only next to tangency,
    where the step's higher derivatives blow up."""
    return 4.0 / 3.0 * np.abs(fd - _fd_tracks(orc, sc, tr, which, k, H / 2))


EPS = 2.0 ** -53


def _close(got, want, s=None, trunc=0.0):
    """1e-6 relative, plus the rounding noise of the central difference: each
    of the two steps carries a few ulps (~ 2 eps |s|) that the difference
    divides by 2h (the h/2 quotient of the truncation estimate twice that),
    plus the truncation estimate."""
    tol = 1e-6 * np.maximum(1.0, np.abs(want)) + trunc
    if s is not None:
        tol = tol + 48 * EPS * np.abs(s) / (2 * H)
    return np.abs(got - want) <= tol


@pytest.mark.parametrize("name,seed", [("diff3", None), ("box4", 0), ("toy8", 1), ("seg4", None),
                                       ("pcon4", None), ("pconm", None)])
def test_adjoint_matches_fd_tracks(orc, name, seed):
    sc = scenes.SCENES[name]() if seed is None else scenes.SCENES[name](seed)
    tr = scenes.sample_tracks(sc, 4000, 41)
    r = orc.navigate(sc, tr)
    ok = _smooth_mask(orc, sc, tr, r)
    adj = orc.adjoint(sc, tr)
    assert np.all(adj["ok"][ok])
    assert ok.mean() > 0.9
    for k in range(3):
        s = r["step"][ok]
        for which, got in (("p", adj["gp"]), ("d", adj["gd"])):
            fd = _fd_tracks(orc, sc, tr, which, k)
            tr_ = _truncation(orc, sc, tr, which, k, fd)
            assert np.all(_close(got[k][ok], fd[ok], s, tr_[ok]))
            # the truncation allowance matters only next to tangency
            assert np.mean(tr_[ok] > 1e-6 * np.maximum(1.0, np.abs(fd[ok])) + 96 * EPS * s / (2 * H)) < 0.005


def _with(sc, **kw):
    d = dict(mother_params=sc.mother_params.copy(), params=sc.params.copy(), trans=sc.trans.copy())
    d.update(kw)
    return scenes.Scene(sc.name, sc.mother_kind, d["mother_params"], sc.kinds, d["params"], sc.rot,
                        d["trans"], sc.pdata)


def _param_slots(kind, row):
    """Row slots that are continuous parameters: all five, but a polycone's
    (sphi, dphi) only (its plane count and table offset are not); the step
    is not differentiable in dphi at a whole turn (a shorter one opens a
    sliver)."""
    if kind == scenes.PCON:
        return (0,) if row[1] >= 2.0 * np.pi else (0, 1)
    return range(5)


@pytest.mark.parametrize("name,seed", [("diff3", None), ("toy8", 1), ("seg4", None), ("pcon4", None),
                                       ("pconm", None)])
def test_adjoint_matches_fd_geometry(orc, name, seed):
    sc = scenes.SCENES[name]() if seed is None else scenes.SCENES[name](seed)
    tr = scenes.sample_tracks(sc, 3000, 42)
    r = orc.navigate(sc, tr)
    ok = _smooth_mask(orc, sc, tr, r)
    adj = orc.adjoint(sc, tr)
    for j in range(sc.n_daughters):
        mine = ok & (adj["winner"] == j)
        other = ok & (adj["winner"] != j)
        for k in range(3):
            tp, tm = sc.trans.copy(), sc.trans.copy()
            tp[j, k] += H
            tm[j, k] -= H
            fd = (orc.navigate(_with(sc, trans=tp), tr)["step"] -
                  orc.navigate(_with(sc, trans=tm), tr)["step"]) / (2 * H)
            assert np.all(_close(adj["gt"][k][mine], fd[mine], r["step"][mine]))
            assert np.all(_close(0.0, fd[other], r["step"][other]))
        for k in _param_slots(sc.kinds[j], sc.params[j]):
            if sc.params[j, k] == 0.0 and not (sc.kinds[j] == scenes.CONE and k in (1, 3)):
                continue
            pp, pm = sc.params.copy(), sc.params.copy()
            pp[j, k] += H
            pm[j, k] -= H
            if pm[j, k] < 0:
                continue
            fd = (orc.navigate(_with(sc, params=pp), tr)["step"] -
                  orc.navigate(_with(sc, params=pm), tr)["step"]) / (2 * H)
            assert np.all(_close(adj["gparams"][k][mine], fd[mine], r["step"][mine])), (j, k)
    mine = ok & (adj["winner"] == -1)
    for k in (range(3) if sc.mother_kind == scenes.BOX else _param_slots(sc.mother_kind, sc.mother_params)):
        if sc.mother_params[k] == 0.0:
            continue
        pp, pm = sc.mother_params.copy(), sc.mother_params.copy()
        pp[k] += H
        pm[k] -= H
        fd = (orc.navigate(_with(sc, mother_params=pp), tr)["step"] -
              orc.navigate(_with(sc, mother_params=pm), tr)["step"]) / (2 * H)
        assert np.all(_close(adj["gparams"][k][mine], fd[mine], r["step"][mine])), k


def test_adjoint_exact_axis_aligned_box(orc):
    """A flat face x_k = c hit along u: s = (c - p_k)/u_k, so ds/dp_k = -1/u_k
    and the other two components vanish."""
    sc = scenes.SCENES["box4"](0)
    tr = scenes.sample_tracks(sc, 4000, 43)
    r = orc.navigate(sc, tr)
    adj = orc.adjoint(sc, tr)
    d = dirs(tr)
    sel = (r["hit"] >= 0) & (r["face"] >= 0) & ((r["second"] - r["step"]) > 1e-6)
    assert sel.sum() > 100
    for i in np.nonzero(sel)[0]:
        ax = int(r["face"][i]) // 2
        want = np.zeros(3)
        want[ax] = -1.0 / d[i, ax]
        assert np.allclose(adj["gp"][:, i], want, rtol=1e-15, atol=0)
