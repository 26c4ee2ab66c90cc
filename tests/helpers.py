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


def tie_band(ref, band=1e-9):
    """Tracks whose second-smallest oracle candidate lies within `band` of the
    winner: their hit index is not unique at that resolution."""
    return (ref["second"] - ref["step"]) < band


def step_tol(ref, floor=1e-9):
    """Per-track step tolerance: max(1e-9 mm, a-priori FP64 error bound)."""
    return np.maximum(floor, ref["err"])
