"""Small shared helpers for the tests (no method arithmetic)."""
import json
import math
import os

import numpy as np

from paper_1312_0816_gb300 import scenes

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def golden(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return json.load(f)


def expr(s):
    return float(eval(s, {"__builtins__": {}}, {"sqrt": math.sqrt, "inf": math.inf, "nan": math.nan,
                                                  "pi": math.pi}))


def scene_from_spec(mother, daughters, name="spec"):
    mk, mp = mother
    rows = [(d[0], d[1], d[2], d[3]) for d in daughters]
    if not rows:
        m = np.zeros(5)
        m[: len(mp)] = mp
        return scenes.Scene(name, int(mk), m, np.zeros(0, np.int32), np.zeros((0, 5)),
                            np.zeros((0, 9)), np.zeros((0, 3)))
    return scenes._scene(name, mk, mp, rows)


def tracks_from(p, d):
    p = np.atleast_2d(np.asarray(p, dtype=np.float64))
    d = np.atleast_2d(np.asarray(d, dtype=np.float64))
    return scenes.Tracks(p[:, 0].copy(), p[:, 1].copy(), p[:, 2].copy(),
                         d[:, 0].copy(), d[:, 1].copy(), d[:, 2].copy())


def points(tr):
    return np.stack([tr.x, tr.y, tr.z], axis=1)


def dirs(tr):
    return np.stack([tr.dx, tr.dy, tr.dz], axis=1)


STEP_TOL = 1e-9   # mm


def step_tol(ref, tracks=None, floor=STEP_TOL):
    """Per-track step tolerance, in units of the step (|d|): max(1e-9 mm, the
    oracle's a-priori FP64 error bound err), err pinned against exact
    crossings in test_oracle_errbound.py."""
    f = floor
    if tracks is not None:
        f = floor / np.sqrt(tracks.dx ** 2 + tracks.dy ** 2 + tracks.dz ** 2)
    return np.maximum(f, ref["err"])


def tie_band(ref, tol=STEP_TOL):
    """Tracks whose second-smallest oracle candidate lies within `tol` of the
    winner: their hit index is not unique at that resolution."""
    return (ref["second"] - ref["step"]) < tol


PERTURB = 1e-9       # mm: start-point moves that define "decided by rounding"
PERTURB_MATCH = 1e-6  # mm: how close the GPU's answer must be to a moved one's


def moved(tracks, k, sign, amount=PERTURB):
    """The tracks with their start points moved by `amount` along axis k."""
    f = [tracks.x.copy(), tracks.y.copy(), tracks.z.copy()]
    f[k] = f[k] + sign * amount
    return scenes.Tracks(*f, tracks.dx, tracks.dy, tracks.dz)


def rounding_decided(orc, scene, tracks, step, hit):
    """Which of these tracks get the GPU's (step, hit) from the oracle for a
    start point moved by 1e-9 mm along some axis: a grazing contact or an edge
    whose outcome FP64 rounding decides (both answers are then correct to
    rounding).  The match is to within max(1e-6 mm, err) of the moved track,
    the hit exact or tie-banded."""
    ok = np.zeros(tracks.n, dtype=bool)
    dn = np.sqrt(tracks.dx ** 2 + tracks.dy ** 2 + tracks.dz ** 2)
    for k in range(3):
        for sg in (-1.0, 1.0):
            r = orc.navigate(scene, moved(tracks, k, sg), nthreads=8)
            tol = np.maximum(PERTURB_MATCH / dn, r["err"])
            same = np.abs(step - r["step"]) <= tol
            ok |= same & ((hit == r["hit"]) | tie_band(r, np.maximum(STEP_TOL / dn, r["err"])))
    return ok


def check_steps(ref, step, hit, tracks=None, max_banded=None, orc=None, scene=None):
    """The parity bar on EVERY track: the step within step_tol() of the
    oracle's, the hit index equal to the oracle's unless the track is
    tie-banded (second candidate within that tolerance of the winner: the
    winner is then decided by rounding), NaN exactly where the oracle's is.
    With the oracle and the scene given, a track outside this bar passes if
    its answer is the oracle's for a start point moved by 1e-9 mm
    (rounding_decided: a grazing contact); those are counted.  max_banded caps
    the share of conditioning-banded tracks (err > 1e-9 mm).  Returns the band
    counts and the largest |dstep| in and out of the conditioning band."""
    step = np.asarray(step)
    hit = np.asarray(hit)
    nan = np.isnan(ref["step"])
    assert np.array_equal(np.isnan(step), nan)
    ok = ~nan
    tol = step_tol(ref, tracks)
    d = np.abs(step - ref["step"])
    tie = ok & tie_band(ref, tol)
    off = ok & (~(d <= tol) | (~tie & (hit != ref["hit"])))
    graze = np.zeros_like(off)
    if off.any() and orc is not None:
        idx = np.nonzero(off)[0]
        sub = scenes.Tracks(*(f[idx] for f in tracks.fields()))
        graze[idx] = rounding_decided(orc, scene, sub, step[idx], hit[idx])
    bad = np.nonzero(off & ~graze)[0]
    assert bad.size == 0, ("step/hit", bad[:8], d[bad[:8]], tol[bad[:8]], hit[bad[:8]], ref["hit"][bad[:8]])
    cond = ok & (ref["err"] > STEP_TOL)
    if max_banded is not None:
        assert cond.mean() <= max_banded, cond.mean()
    return {"n": int(ok.sum()), "tie_banded": int(tie.sum()), "cond_banded": int(cond.sum()),
            "rounding_decided": int(graze.sum()),
            "hit_differs_in_tie_band": int((tie & (hit != ref["hit"])).sum()),
            "max_dstep": float(d[ok & ~cond & ~graze].max(initial=0.0)),
            "max_dstep_cond_banded": float(d[cond & ~graze].max(initial=0.0))}
