"""Gradients of the navigator step (adjoint kernel) on the GPU.

Checked against the oracle's adjoint (the same implicit-function rule written
independently), against central finite differences of the GPU forward step
(h = 1e-6 mm), for the geometry sums against finite differences of rebuilt
volumes, for determinism, and through torch.autograd.  Tracks near a kink
(the winner or its surface changes under a 1e-3 mm move, or a tie within
1e-3 mm) are excluded: the step is not differentiable there.
"""
import numpy as np
import pytest

from helpers import points, dirs, tracks_from
from paper_1312_0816_gb300 import scenes

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

H = 1e-6
EPS = 2.0 ** -53


@pytest.fixture(scope="module")
def g():
    import paper_1312_0816_gb300 as pkg

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    pkg.load()
    return pkg


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def smooth_mask(orc, sc, tr, ref):
    """Tracks whose winner and crossed surface stay the same under moves of
    the start point by 1e-3 mm and of the direction by 1e-5 along every
    axis, with no other candidate within 1e-2 mm of the step."""
    ok = (ref["second"] - ref["step"]) > 1e-2
    ok &= ref["hit"] >= -1
    p, d = points(tr), dirs(tr)
    for k in range(3):
        for sg in (-1.0, 1.0):
            for which, size in (("p", 1e-3), ("d", 1e-5)):
                q = (p if which == "p" else d).copy()
                q[:, k] += sg * size
                moved = tracks_from(q, d) if which == "p" else tracks_from(p, q)
                rr = orc.navigate(sc, moved, nthreads=8)
                ok &= (rr["hit"] == ref["hit"]) & (rr["face"] == ref["face"])
    return ok


def forward(g, vol, tr, mode=0):
    s, h = g.geo_dist_to_boundary(vol, *(dev(f) for f in tr.fields()), mode=mode)
    torch.cuda.synchronize()
    return s, h


def close(got, want, err, trunc, rel=1e-6):
    """Central difference vs the adjoint: each forward step is within about
    twice the oracle's a-priori bound `err` of the exact one, so the
    difference quotient carries up to 2 err / H of rounding; `trunc` is the
    difference quotient's own truncation error, estimated from a second
    quotient at H/2 (large only next to tangency, where the step's higher
    derivatives blow up)."""
    tol = rel * np.maximum(1.0, np.abs(want)) + 2.0 * err / H + trunc
    return np.abs(got - want) <= tol


def central(fstep, base, k, h):
    a, b = base.copy(), base.copy()
    a[:, k] += h
    b[:, k] -= h
    return (fstep(a) - fstep(b)) / (2 * h)


@pytest.mark.parametrize("name,n", [("box4", 1 << 18), ("diff3", 1 << 16), ("toy8", 1 << 16), ("seg4", 1 << 16),
                                    ("pcon4", 1 << 16), ("pconm", 1 << 16)])
def test_track_gradients(g, orc, name, n):
    sc = scenes.SCENES[name]()
    vol = g.geo_build_volume(sc)
    tr = scenes.sample_tracks(sc, n, 41)
    ref = orc.navigate(sc, tr, nthreads=8)
    ok = smooth_mask(orc, sc, tr, ref)
    adj = orc.adjoint(sc, tr)
    ok &= adj["ok"]
    assert ok.mean() > 0.9
    s, h = forward(g, vol, tr)
    x = [dev(f) for f in tr.fields()]
    ones = torch.ones(n, dtype=torch.float64, device="cuda")
    gp, gd = g.geo_dist_to_boundary_adjoint(vol, *x, h, ones, want_geometry=False)
    gp, gd = gp.cpu().numpy(), gd.cpu().numpy()
    # the oracle's adjoint (independent code, same rule)
    assert np.allclose(gp[:, ok], adj["gp"][:, ok], rtol=1e-8, atol=1e-9)
    assert np.allclose(gd[:, ok], adj["gd"][:, ok], rtol=1e-8, atol=1e-7)
    # central differences of the GPU forward step
    err = np.maximum(ref["err"], 16 * EPS * np.abs(ref["step"]))
    p, d = points(tr), dirs(tr)
    for k in range(3):
        for which, base in (("p", p), ("d", d)):
            def fstep(q):
                t = tracks_from(q, d) if which == "p" else tracks_from(p, q)
                return forward(g, vol, t)[0].cpu().numpy()

            fd = central(fstep, base, k, H)
            fd2 = central(fstep, base, k, H / 2)
            # truncation of the H quotient ~ 4/3 of its difference to the H/2
            # one, plus the rounding the H/2 quotient adds to that difference
            trunc = 4.0 / 3.0 * np.abs(fd - fd2) + 4.0 * err / H
            got = (gp if which == "p" else gd)[k]
            bad = ~close(got[ok], fd[ok], err[ok], trunc[ok])
            assert not bad.any(), (which, k, int(bad.sum()))
            # truncation above the rounding noise is rare (next to tangency)
            big = 4.0 / 3.0 * np.abs(fd - fd2) > 1e-6 * np.maximum(1.0, np.abs(fd)) + 8.0 * err / H
            assert np.mean(big[ok]) < 0.01


def _scene_with(sc, trans=None, params=None, mparams=None):
    return scenes.Scene(sc.name, sc.mother_kind, sc.mother_params if mparams is None else mparams, sc.kinds,
                        sc.params if params is None else params, sc.rot, sc.trans if trans is None else trans,
                        sc.pdata)


def _slots(kind, row):
    """Continuous parameter slots of a row: a polycone's (sphi, dphi) only, and
    no dphi at a whole turn (a shorter turn opens a sliver)."""
    if kind == scenes.PCON:
        return (0,) if row[1] >= 2 * np.pi else (0, 1)
    return range(5)


@pytest.mark.parametrize("name,n", [("box4", 1 << 18), ("diff3", 1 << 16), ("seg4", 1 << 16), ("pcon4", 1 << 16),
                                    ("pconm", 1 << 16)])
def test_geometry_gradients_match_fd(g, orc, name, n):
    """d(sum over smooth tracks of step)/d(translations, shape parameters)."""
    sc = scenes.SCENES[name]()
    vol = g.geo_build_volume(sc)
    tr = scenes.sample_tracks(sc, n, 42)
    ref = orc.navigate(sc, tr, nthreads=8)
    ok = smooth_mask(orc, sc, tr, ref)
    adj = orc.adjoint(sc, tr)
    ok &= adj["ok"]
    mask = ok.astype(np.float64)
    s, h = forward(g, vol, tr)
    x = [dev(f) for f in tr.fields()]
    gp, gd, gt, gprm = g.geo_dist_to_boundary_adjoint(vol, *x, h, dev(mask))
    gt, gprm = gt.cpu().numpy(), gprm.cpu().numpy()
    # the same sums from the oracle's per-track adjoint
    for j in range(sc.n_daughters):
        sel = ok & (adj["winner"] == j)
        assert np.allclose(gt[j], adj["gt"][:, sel].sum(axis=1), rtol=1e-9, atol=1e-9)
        assert np.allclose(gprm[j], adj["gparams"][:, sel].sum(axis=1), rtol=1e-9, atol=1e-9)
    sel = ok & (adj["winner"] == -1)
    assert np.allclose(gprm[sc.n_daughters], adj["gparams"][:, sel].sum(axis=1), rtol=1e-9, atol=1e-9)

    def steps(scene):
        return forward(g, g.geo_build_volume(scene), tr)[0].cpu().numpy()

    def fd_of(plus, minus):
        # per-track differences first, so no large totals cancel
        return float(((steps(plus) - steps(minus)) * mask).sum()) / (2 * H)

    # each step within about twice the a-priori bound of the exact one
    err = np.maximum(ref["err"], 16 * EPS * np.abs(ref["step"]))
    noise = 2.0 * float(err[ok].sum()) / H
    for j in range(sc.n_daughters):
        for k in range(3):
            tp, tm = sc.trans.copy(), sc.trans.copy()
            tp[j, k] += H
            tm[j, k] -= H
            fd = fd_of(_scene_with(sc, trans=tp), _scene_with(sc, trans=tm))
            assert abs(fd - gt[j, k]) <= 1e-6 * max(1.0, abs(fd)) + noise, (j, k, fd, gt[j, k])
        for k in _slots(sc.kinds[j], sc.params[j]):
            if sc.params[j, k] == 0.0:
                continue
            if sc.kinds[j] == scenes.TUBS and k == 4 and sc.params[j, 4] + H > 2 * np.pi:
                continue   # a whole turn cannot grow
            pp, pm = sc.params.copy(), sc.params.copy()
            pp[j, k] += H
            pm[j, k] -= H
            fd = fd_of(_scene_with(sc, params=pp), _scene_with(sc, params=pm))
            assert abs(fd - gprm[j, k]) <= 1e-6 * max(1.0, abs(fd)) + noise, (j, k, fd, gprm[j, k])
    nd = sc.n_daughters
    for k in _slots(sc.mother_kind, sc.mother_params):
        if sc.mother_params[k] == 0.0:
            continue
        mp, mm = sc.mother_params.copy(), sc.mother_params.copy()
        mp[k] += H
        mm[k] -= H
        fd = fd_of(_scene_with(sc, mparams=mp), _scene_with(sc, mparams=mm))
        assert abs(fd - gprm[nd, k]) <= 1e-6 * max(1.0, abs(fd)) + noise, ("mother", k, fd, gprm[nd, k])


def test_adjoint_is_deterministic(g):
    sc = scenes.grid512(5)
    vol = g.geo_build_volume(sc, voxelize=True)
    tr = scenes.sample_tracks(sc, 1 << 18, 43)
    s, h = forward(g, vol, tr, mode=1)
    x = [dev(f) for f in tr.fields()]
    w = torch.rand(tr.n, dtype=torch.float64, device="cuda")
    a = g.geo_dist_to_boundary_adjoint(vol, *x, h, w)
    b = g.geo_dist_to_boundary_adjoint(vol, *x, h, w)
    for u, v in zip(a, b):
        assert torch.equal(u, v)


def test_autograd_function(g):
    from paper_1312_0816_gb300.autograd import dist_to_boundary

    sc = scenes.diff3()
    vol = g.geo_build_volume(sc)
    tr = scenes.sample_tracks(sc, 5000, 44)
    p = torch.stack([dev(tr.x), dev(tr.y), dev(tr.z)]).requires_grad_(True)
    d = torch.stack([dev(tr.dx), dev(tr.dy), dev(tr.dz)]).requires_grad_(True)
    trans = torch.from_numpy(sc.trans.copy()).cuda().requires_grad_(True)
    params = torch.from_numpy(np.vstack([sc.params, sc.mother_params])).cuda().requires_grad_(True)
    step, hit = dist_to_boundary(vol, p, d, trans, params, mode=1)
    w = torch.linspace(0.5, 1.5, tr.n, dtype=torch.float64, device="cuda")
    (step * w).sum().backward()
    gp, gd, gt, gprm = g.geo_dist_to_boundary_adjoint(vol, p[0].detach(), p[1].detach(), p[2].detach(),
                                                      d[0].detach(), d[1].detach(), d[2].detach(), hit, w)
    assert torch.equal(p.grad, gp) and torch.equal(d.grad, gd)
    assert torch.equal(trans.grad, gt) and torch.equal(params.grad, gprm)
