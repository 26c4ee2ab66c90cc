"""Pins the oracle's a-priori FP64 error bound `err` of a navigator step.

The GPU parity tests compare steps at max(1e-9 mm, err) and count the
tracks whose err exceeds 1e-9 mm; err must therefore really bound what FP64
rounding does to a step.  Here it is checked against the exact answer for
the given FP64 inputs: the crossing of the winning surface computed in
212-bit arithmetic (tests/exact_root.py), for

* the oracle's own step (exact roots on FP64 local coordinates), and
* a deliberately plain binary64 evaluation of the same crossing (transform
  summed in another order, textbook quadratic formula with B*B - A*C): a
  stand-in for any FP64 implementation, the GPU's included,

on random rays, the adversarial rays (grazing planes, box edges and corners,
cylinder and cone tangents, rims, apexes, polycone sections and phi faces)
and rays whose direction is not a unit vector.  Both must lie within err/2 of
the exact crossing, so that two FP64 implementations differ by at most err.
The bound must not be vacuous either: on every scene some track comes within
a factor of 100 of it.  Sec. 3.2 cross-checks the vector navigator against
the scalar one on every track; this is what makes such a check precise.
"""
import contextlib
import subprocess

import numpy as np
import pytest

from exact_root import exact_root, plain_root
from paper_1312_0816_gb300 import scenes

SCENES = {
    "box4": lambda: scenes.box4(0),
    "toy40": lambda: scenes.toy40(1),
    "diff3": lambda: scenes.diff3(),
    "seg4": lambda: scenes.seg4(),
    "pcon4": lambda: scenes.pcon4(),
    "pconm": lambda: scenes.pconm(),
    "grid512": lambda: scenes.grid512(5),
}


def nonunit(sc, n, seed):
    """Random rays with |d| log-uniform in [1e-3, 1e3] (steps in units of |d|)."""
    tr = scenes.sample_tracks(sc, n, seed)
    f = 10.0 ** np.random.default_rng(seed + 7).uniform(-3.0, 3.0, n)
    return scenes.Tracks(tr.x, tr.y, tr.z, tr.dx * f, tr.dy * f, tr.dz * f)


def ratios(sc, tr, ref, chains=None, composed=False):
    """|step - exact| / err for the oracle and for the plain evaluation, over
    the tracks with a finite step and a winning surface."""
    ro, rp = [], []
    for i in range(tr.n):
        s, h, f, e = ref["step"][i], int(ref["hit"][i]), int(ref["face"][i]), ref["err"][i]
        if not np.isfinite(s) or h < -1 or f < 0:
            continue
        p = (tr.x[i], tr.y[i], tr.z[i])
        d = (tr.dx[i], tr.dy[i], tr.dz[i])
        ch = chains[i] if chains is not None else ()
        vol = sc[i] if isinstance(sc, list) else sc
        se, _ = exact_root(vol, h, f, p, d, s, ch)
        sp = plain_root(vol, h, f, p, d, s, ch, composed)
        assert np.isfinite(se) and np.isfinite(sp), i
        ro.append(abs(s - se) / e)
        rp.append(abs(sp - se) / e)
    return np.array(ro), np.array(rp)


@pytest.mark.parametrize("name", list(SCENES))
def test_err_bounds_the_fp64_error(orc, name):
    sc = SCENES[name]()
    worst = 0.0
    for kind, tr in (("random", scenes.sample_tracks(sc, 600, 3)),
                     ("adversarial", scenes.adversarial_tracks(sc, 600, 4)),
                     ("non-unit d", nonunit(sc, 300, 5))):
        ref = orc.navigate(sc, tr, nthreads=4)
        ro, rp = ratios(sc, tr, ref)
        assert ro.size > 0.9 * tr.n, (kind, ro.size)
        assert ro.max() <= 0.5, (kind, "oracle", ro.max())
        assert rp.max() <= 0.5, (kind, "plain FP64", rp.max())
        worst = max(worst, rp.max())
        if kind == "random":
            # err > 1e-9 mm is the conditioning band: rare on random rays
            assert np.mean(ref["err"] > 1e-9) <= 1e-3
    assert worst >= 0.01, worst


@contextlib.contextmanager
def planted(orc, tmp_path, old, new):
    """The oracle built from its source with one edit (a planted mistake),
    loaded in place of the real one for the duration."""
    src = open(orc._SRC).read()
    assert src.count(old) == 1, old
    c = tmp_path / "planted.c"
    c.write_text(src.replace(old, new))
    so = tmp_path / "planted.so"
    subprocess.check_call(["gcc", *orc.CFLAGS, str(c), "-o", str(so), "-lm", "-lpthread"])
    saved = orc._lib, orc._LIB_PATH
    orc._lib, orc._LIB_PATH = None, str(so)
    try:
        yield orc
    finally:
        orc._lib, orc._LIB_PATH = saved


# each plausible slip in the bound and a track set on which the check above
# then fails
PLANTS = {
    "no division by |d|": ("* cond / dn +", "* cond +", "grid512", "nonunit"),
    "quadric rounding term dropped": ("16.0 * qcoef", "0.0 * qcoef", "grid512", "random"),
    "incidence factor dropped": ("if (c2 > cond) cond = c2;", "", "diff3", "adversarial"),
}


@pytest.mark.parametrize("plant", list(PLANTS))
def test_err_check_catches_a_planted_mistake(orc, tmp_path, plant):
    old, new, name, kind = PLANTS[plant]
    sc = SCENES[name]()
    tr = {"random": lambda: scenes.sample_tracks(sc, 2000, 3),
          "adversarial": lambda: scenes.adversarial_tracks(sc, 600, 4),
          "nonunit": lambda: nonunit(sc, 300, 5)}[kind]()
    with planted(orc, tmp_path, old, new) as bad:
        ref = bad.navigate(sc, tr, nthreads=4)
    ro, rp = ratios(sc, tr, ref)
    assert max(ro.max(), rp.max()) > 0.5


def _chains(w, nodes_tab, node):
    """Placements (R, t) from the root down to each node."""
    out = []
    for m in node:
        ch = []
        while m > 0:
            par = nodes_tab["parent"][m]
            v = w.volumes[nodes_tab["lv"][par]]
            j = nodes_tab["slot"][m]
            ch.append((v.rot[j], v.trans[j]))
            m = par
        out.append(ch[::-1])
    return out


@pytest.mark.parametrize("make", [scenes.world_toy, scenes.world_pcon], ids=["toy", "pcon"])
def test_world_step_err_bounds_the_fp64_error(orc, make):
    """The geometry-tree step: err includes the rounding of the placements
    that bring a world point into its node, and bounds the step's error for
    the oracle (one level after another), for a plain evaluation level by
    level and for one through the composed world transform of the node (as
    the GPU does), over three steps of transport."""
    w = make()
    tab = orc.world_nodes(w)
    tr = scenes.world_points(w, 400, 11)
    node = orc.world_locate(w, tr)
    flag = np.full(tr.n, -1, dtype=np.int32)
    checked = 0
    for _ in range(3):
        alive = node >= 0
        s, nn, fl, info = orc.world_step(w, tr, node, flag, info=True)
        idx = np.nonzero(alive & (info["hit"] >= -1))[0]
        sub = scenes.Tracks(*(f[idx] for f in tr.fields()))
        ref = {"step": s[idx], "hit": info["hit"][idx], "face": info["face"][idx], "err": info["err"][idx]}
        vols = [w.volumes[tab["lv"][m]] for m in node[idx]]
        ch = _chains(w, tab, node[idx])
        ro, rp = ratios(vols, sub, ref, ch)
        _, rc = ratios(vols, sub, ref, ch, composed=True)
        assert ro.max() <= 0.5 and rp.max() <= 0.5 and rc.max() <= 0.5, (ro.max(), rp.max(), rc.max())
        checked += ro.size
        st = np.where(alive, s, 0.0)
        tr = scenes.Tracks(tr.x + st * tr.dx, tr.y + st * tr.dy, tr.z + st * tr.dz, tr.dx, tr.dy, tr.dz)
        node = np.where(alive, nn, -1).astype(np.int32)
        flag = np.where(alive, fl, -1).astype(np.int32)
    assert checked > 400
