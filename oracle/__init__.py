"""CPU oracle for the vector navigator -- TEST INFRASTRUCTURE.

Only `tests/`, `__graft_entry__.smoke()` and the CPU-baseline leg of
`bench.py` may import this package.  The product path never calls it.

The arithmetic lives in `geo_oracle.c` (plain scalar FP64 C, compiled with
-O2 -ffp-contract=off).  This module only compiles it with gcc and marshals
numpy arrays through ctypes.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "geo_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "libgeo_oracle.so")
_lib = None

CFLAGS = ["-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared", "-std=c11"]


def build(force: bool = False) -> str:
    """Compile the oracle with gcc into oracle/_build (idempotent)."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", *CFLAGS, _SRC, "-o", tmp, "-lm", "-lpthread"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB_PATH)
        dp = ctypes.POINTER(ctypes.c_double)
        ip = ctypes.POINTER(ctypes.c_int32)
        scene = [ctypes.c_int, dp, ctypes.c_int, ip, dp, dp, dp, dp]
        L.orc_navigate.argtypes = scene + [ctypes.c_int64] + [dp] * 6 + [dp, ip, dp, dp, ip, ctypes.c_int]
        L.orc_navigate.restype = None
        L.orc_contains_nav.argtypes = scene + [ctypes.c_int64, dp, dp, dp, ip, ctypes.c_int]
        L.orc_contains_nav.restype = None
        L.orc_safety_nav.argtypes = scene + [ctypes.c_int64, dp, dp, dp, dp, ctypes.c_int]
        L.orc_safety_nav.restype = None
        L.orc_safety_estimate_nav.argtypes = scene + [ctypes.c_int64, dp, dp, dp, dp, ctypes.c_int]
        L.orc_safety_estimate_nav.restype = None
        L.orc_adjoint.argtypes = scene + [ctypes.c_int64] + [dp] * 6 + [dp, dp, ip, dp, dp, ip]
        L.orc_adjoint.restype = None
        L.orc_shape_batch.argtypes = [ctypes.c_int, dp, dp, ctypes.c_int64, dp, dp, ctypes.c_int, dp, ip]
        L.orc_shape_batch.restype = None
        L.orc_shape_batch_err.argtypes = [ctypes.c_int, dp, dp, ctypes.c_int64, dp, dp, ctypes.c_int, ctypes.c_double,
                                          dp, dp]
        L.orc_shape_batch_err.restype = None
        world = [ctypes.c_int, ip, dp, ip, ip, ip, dp, dp, dp, ip, dp, ctypes.c_int, ctypes.c_int, ip, ip, ip, ip]
        L.orc_world_nodes.argtypes = world
        L.orc_world_nodes.restype = ctypes.c_int
        L.orc_world_locate.argtypes = world + [ctypes.c_int64, dp, dp, dp, ip]
        L.orc_world_locate.restype = ctypes.c_int
        L.orc_world_step.argtypes = world + [ctypes.c_int64] + [dp] * 6 + [ip, ip, dp, ip, ip, dp, ip, ip]
        L.orc_world_step.restype = ctypes.c_int
        _lib = L
    return _lib


def _d(a):
    a = np.ascontiguousarray(a, dtype=np.float64)
    return a, a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _i(a):
    a = np.ascontiguousarray(a, dtype=np.int32)
    return a, a.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))


def _scene_args(scene):
    keep = []
    mp, mpp = _d(scene.mother_params)
    k, kp = _i(scene.kinds)
    pr, prp = _d(scene.params.reshape(-1))
    ro, rop = _d(scene.rot.reshape(-1))
    tr, trp = _d(scene.trans.reshape(-1))
    pd, pdp = _d(np.concatenate([np.asarray(scene.pdata, dtype=np.float64), [0.0]]))
    keep += [mp, k, pr, ro, tr, pd]
    return keep, [int(scene.mother_kind), mpp, int(scene.n_daughters), kp, prp, rop, trp, pdp]


def _track_args(tracks, fields=6):
    keep, ptrs = [], []
    for f in tracks.fields()[:fields]:
        a, p = _d(f)
        keep.append(a)
        ptrs.append(p)
    return keep, ptrs


def navigate(scene, tracks, nthreads: int = 1):
    """Fig. 1 navigator over a basket.  Returns dict with step, hit, second
    (second-smallest candidate), err (a-priori FP64 error bound), face."""
    n = tracks.n
    ks, sargs = _scene_args(scene)
    kt, targs = _track_args(tracks)
    step = np.empty(n)
    hit = np.empty(n, dtype=np.int32)
    second = np.empty(n)
    err = np.empty(n)
    face = np.empty(n, dtype=np.int32)
    lib().orc_navigate(*sargs, n, *targs, _d(step)[1], _i(hit)[1], _d(second)[1], _d(err)[1],
                       _i(face)[1], int(nthreads))
    return {"step": step, "hit": hit, "second": second, "err": err, "face": face}


def contains(scene, tracks, nthreads: int = 1):
    n = tracks.n
    ks, sargs = _scene_args(scene)
    kt, targs = _track_args(tracks, 3)
    where = np.empty(n, dtype=np.int32)
    lib().orc_contains_nav(*sargs, n, *targs, _i(where)[1], int(nthreads))
    return where


def safety(scene, tracks, nthreads: int = 1):
    n = tracks.n
    ks, sargs = _scene_args(scene)
    kt, targs = _track_args(tracks, 3)
    out = np.empty(n)
    lib().orc_safety_nav(*sargs, n, *targs, _d(out)[1], int(nthreads))
    return out


def safety_estimate(scene, tracks, nthreads: int = 1):
    """The under-estimating safety: min of the mother's and daughters' simpler
    bounds (see geo_oracle.c); never above the exact safety."""
    n = tracks.n
    ks, sargs = _scene_args(scene)
    kt, targs = _track_args(tracks, 3)
    out = np.empty(n)
    lib().orc_safety_estimate_nav(*sargs, n, *targs, _d(out)[1], int(nthreads))
    return out


def adjoint(scene, tracks):
    """Per-track gradient of the step: dp (3,n), dd (3,n), winner index, the
    winner's dt (3,n) and dparams (5,n), ok flag."""
    n = tracks.n
    ks, sargs = _scene_args(scene)
    kt, targs = _track_args(tracks)
    gp = np.empty(3 * n)
    gd = np.empty(3 * n)
    gt = np.empty(3 * n)
    gprm = np.empty(5 * n)
    win = np.empty(n, dtype=np.int32)
    ok = np.empty(n, dtype=np.int32)
    lib().orc_adjoint(*sargs, n, *targs, _d(gp)[1], _d(gd)[1], _i(win)[1], _d(gt)[1], _d(gprm)[1],
                      _i(ok)[1])
    return {"gp": gp.reshape(3, n), "gd": gd.reshape(3, n), "winner": win,
            "gt": gt.reshape(3, n), "gparams": gprm.reshape(5, n), "ok": ok.astype(bool)}


_WHAT = {"dist_out": 0, "dist_in": 1, "contains": 2, "safety_out": 3, "safety_in": 4}


def shape(kind: int, params, x, u=None, what: str = "dist_out"):
    """One solid in its own frame; x, u are (n, 3); params is its row, or a
    polycone spec (an object with z, rmin, rmax, sphi, dphi).  Returns values
    (and the hit face for the two distance queries)."""
    p = np.zeros(5)
    planes = np.zeros(1)
    if hasattr(params, "rmax"):
        planes = np.concatenate([np.asarray(params.z, float), np.asarray(params.rmin, float),
                                 np.asarray(params.rmax, float)])
        p[:4] = (params.sphi, params.dphi, len(params.z), 0)
    else:
        p[: len(params)] = params
    x = np.ascontiguousarray(np.asarray(x, dtype=np.float64).reshape(-1, 3))
    n = x.shape[0]
    u = np.zeros_like(x) if u is None else np.ascontiguousarray(np.asarray(u, dtype=np.float64).reshape(-1, 3))
    out = np.empty(n)
    face = np.empty(n, dtype=np.int32)
    pa, pp = _d(p)
    pl, plp = _d(planes)
    lib().orc_shape_batch(int(kind), pp, plp, n, _d(x)[1], _d(u)[1], _WHAT[what], _d(out)[1], _i(face)[1])
    if what in ("dist_out", "dist_in"):
        return out, face
    return out


def shape_err(kind: int, params, x, u, what: str = "dist_out", tnorm: float = 0.0):
    """For a distance query of one solid: the answer's a-priori FP64 error
    bound (tnorm: distance of the solid's placement from the frame the query
    was posed in) and the gap to the nearest crossing of another of its
    surfaces.  Returns (err, gap)."""
    p = np.zeros(5)
    planes = np.zeros(1)
    if hasattr(params, "rmax"):
        planes = np.concatenate([np.asarray(params.z, float), np.asarray(params.rmin, float),
                                 np.asarray(params.rmax, float)])
        p[:4] = (params.sphi, params.dphi, len(params.z), 0)
    else:
        p[: len(params)] = params
    x = np.ascontiguousarray(np.asarray(x, dtype=np.float64).reshape(-1, 3))
    u = np.ascontiguousarray(np.asarray(u, dtype=np.float64).reshape(-1, 3))
    n = x.shape[0]
    err = np.empty(n)
    gap = np.empty(n)
    pa, pp = _d(p)
    pl, plp = _d(planes)
    lib().orc_shape_batch_err(int(kind), pp, plp, n, _d(x)[1], _d(u)[1], _WHAT[what], float(tnorm), _d(err)[1],
                              _d(gap)[1])
    return err, gap


MAX_NODES = 1 << 20


def _world_args(world, max_nodes=MAX_NODES):
    f = world.flat()
    keep, args = [], []
    nlv = len(world.volumes)
    f["pdata"] = np.concatenate([f["pdata"], [0.0]])
    for key, conv in (("mkind", _i), ("mparams", _d), ("nd", _i), ("doff", _i), ("kinds", _i), ("params", _d),
                      ("rot", _d), ("trans", _d), ("child", _i), ("pdata", _d)):
        a, ptr = conv(np.asarray(f[key]).reshape(-1))
        keep.append(a)
        args.append(ptr)
    table = [np.zeros(max_nodes, dtype=np.int32) for _ in range(4)]
    keep += table
    return keep, table, [nlv] + args + [f["root"], max_nodes] + [_i(t)[1] for t in table]


def world_nodes(world):
    """Breadth-first node table: dict of lv, parent, slot, first (child)."""
    keep, table, args = _world_args(world)
    nn = lib().orc_world_nodes(*args)
    assert nn > 0
    return {k: t[:nn].copy() for k, t in zip(("lv", "parent", "slot", "first"), table)}


def world_locate(world, tracks):
    """Node of every point (-1 outside the root, -2 non-finite)."""
    keep, table, args = _world_args(world)
    kt, targs = _track_args(tracks, 3)
    node = np.empty(tracks.n, dtype=np.int32)
    assert lib().orc_world_locate(*args, tracks.n, *targs, _i(node)[1]) > 0
    return node


def world_step(world, tracks, node_in, blocked_in=None, info=False):
    """The step of Fig. 1 in each track's node, then the track's node after
    the step (-1 left the root, -2 not inside its node or invalid) and its
    flag: j >= 0 = daughter j of the node was just left (its re-entry
    distance replaces DistFromOutside), -2 = the node was just entered
    through its surface, -1 = none (after Locate).  Returns step, node,
    flag, and with info=True a dict of the step's a-priori FP64 error bound
    (err, the node's placements included), the winner in the node's volume
    (hit) and its surface (face)."""
    keep, table, args = _world_args(world)
    kt, targs = _track_args(tracks)
    nin, nptr = _i(node_in)
    if blocked_in is None:
        blocked_in = np.full(tracks.n, -1, dtype=np.int32)
    bin_, bptr = _i(blocked_in)
    step = np.empty(tracks.n)
    node = np.empty(tracks.n, dtype=np.int32)
    blk = np.empty(tracks.n, dtype=np.int32)
    err = np.empty(tracks.n)
    hit = np.empty(tracks.n, dtype=np.int32)
    face = np.empty(tracks.n, dtype=np.int32)
    assert lib().orc_world_step(*args, tracks.n, *targs, nptr, bptr, _d(step)[1], _i(node)[1], _i(blk)[1],
                                _d(err)[1], _i(hit)[1], _i(face)[1]) > 0
    if info:
        return step, node, blk, {"err": err, "hit": hit, "face": face}
    return step, node, blk
