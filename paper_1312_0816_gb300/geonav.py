"""Thin Python binding of the C ABI in include/geo.h (libgeonav.so).

Each function carries the C name and only marshals arguments: torch CUDA
tensors become device pointers, the current torch stream becomes the
cudaStream_t.  All navigation work runs in the library's CUDA kernels; there
is no CPU path.  If the library cannot be loaded the call raises.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build_lib

GEO_OK = 0
GEO_FP64 = 0
GEO_FP32_REFINE = 1
GEO_SAFETY_ESTIMATE = 2   # geo_safety only: the cheaper under-estimate
GEO_BOX, GEO_TUBE, GEO_CONE, GEO_TUBS, GEO_PCON = 0, 1, 2, 3, 4
GEO_MAX_PLANES = 32
GEO_TILE_TRACKS = 384   # include/geo.h: tracks per tile of the filter kernels and batched launches

_STATUS = {0: "GEO_OK", 1: "GEO_ERR_INVALID_ARG", 2: "GEO_ERR_SHAPE_PARAMS", 3: "GEO_ERR_OOM",
           4: "GEO_ERR_CUDA", 5: "GEO_ERR_DEVICE_ASSERT", 6: "GEO_ERR_UNSUPPORTED"}


class GeoError(RuntimeError):
    def __init__(self, status: int, what: str):
        self.status = status
        super().__init__(f"{what}: {_STATUS.get(status, status)} ({geo_status_string(status)})")


class geo_placed_shape(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("reserved", ctypes.c_int32), ("p", ctypes.c_double * 5),
                ("rot", ctypes.c_double * 9), ("trans", ctypes.c_double * 3),
                ("planes", ctypes.POINTER(ctypes.c_double))]


class geo_build_opts(ctypes.Structure):
    _fields_ = [("voxelize", ctypes.c_int32), ("grid", ctypes.c_int32 * 3)]


class geo_basket(ctypes.Structure):
    _fields_ = [("volume", ctypes.c_int32), ("reserved", ctypes.c_int32), ("offset", ctypes.c_int64),
                ("count", ctypes.c_int64)]


class geo_batch_opts(ctypes.Structure):
    _fields_ = [("tile_order", ctypes.c_int32), ("blocks_per_sm", ctypes.c_int32), ("tile_tracks", ctypes.c_int32)]


_lib = None
EXPORTS = ("geo_build_volume", "geo_destroy_volume", "geo_volume_info", "geo_dist_to_boundary",
           "geo_contains", "geo_safety", "geo_dist_to_boundary_host", "geo_dist_to_boundary_stats",
           "geo_check_device_status", "geo_probe_pipe", "geo_build_batch", "geo_destroy_batch",
           "geo_dist_to_boundary_batched", "geo_dist_to_boundary_batched_noalloc", "geo_adjoint_workspace_size",
           "geo_dist_to_boundary_adjoint", "geo_shape_query", "geo_build_world", "geo_destroy_world",
           "geo_world_info", "geo_world_nodes", "geo_world_locate", "geo_world_step", "geo_selftest_wait_timeout",
           "geo_debug_fail_alloc", "geo_status_string")


def library_path() -> str:
    return build_lib.LIB


def load(build_if_stale: bool = True):
    """Loads libgeonav.so (compiling it first if it is missing or stale)."""
    global _lib
    if _lib is not None:
        return _lib
    if build_if_stale and not build_lib.up_to_date():
        build_lib.build()
    if not os.path.exists(build_lib.LIB):
        raise RuntimeError(f"libgeonav.so not found at {build_lib.LIB}; run __graft_entry__.build()")
    L = ctypes.CDLL(build_lib.LIB)
    vp, dp, ip = ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p
    i32, i64 = ctypes.c_int32, ctypes.c_int64
    L.geo_build_volume.argtypes = [ctypes.POINTER(geo_placed_shape), ctypes.POINTER(geo_placed_shape), i32,
                                   ctypes.POINTER(geo_build_opts), vp, ctypes.POINTER(vp)]
    L.geo_destroy_volume.argtypes = [vp]
    L.geo_volume_info.argtypes = [vp, ctypes.POINTER(i32), ctypes.POINTER(i32), ctypes.POINTER(i32 * 3)]
    L.geo_dist_to_boundary.argtypes = [vp, dp, dp, dp, dp, dp, dp, i64, dp, ip, dp, i32, vp]
    L.geo_contains.argtypes = [vp, dp, dp, dp, i64, ip, i32, vp]
    L.geo_safety.argtypes = [vp, dp, dp, dp, i64, dp, i32, vp]
    L.geo_build_world.argtypes = [ctypes.POINTER(vp), i32, ctypes.POINTER(ctypes.c_int32), i32, vp, ctypes.POINTER(vp)]
    L.geo_destroy_world.argtypes = [vp]
    L.geo_world_info.argtypes = [vp, ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int32)]
    L.geo_world_nodes.argtypes = [vp] + [ctypes.POINTER(ctypes.c_int32)] * 4
    L.geo_world_locate.argtypes = [vp, dp, dp, dp, i64, ip, vp]
    L.geo_world_step.argtypes = [vp, dp, dp, dp, dp, dp, dp, i64, ip, ip, dp, ip, ip, i32, vp]
    L.geo_shape_query.argtypes = [ctypes.POINTER(geo_placed_shape), i32, dp, dp, dp, dp, dp, dp, i64, dp, ip, vp]
    L.geo_dist_to_boundary_host.argtypes = [vp, dp, dp, dp, dp, dp, dp, i64, dp, ip, i32, i64, vp]
    L.geo_dist_to_boundary_stats.argtypes = [vp, dp, dp, dp, dp, dp, dp, i64, dp, ip, ip, vp]
    L.geo_check_device_status.argtypes = [vp, ctypes.POINTER(ctypes.c_uint32), vp]
    L.geo_probe_pipe.argtypes = [i32, i64, i32, vp, vp, ctypes.POINTER(ctypes.c_double)]
    L.geo_build_batch.argtypes = [ctypes.POINTER(vp), i32, ctypes.POINTER(geo_basket), i32,
                                  ctypes.POINTER(geo_batch_opts), vp, ctypes.POINTER(vp)]
    L.geo_destroy_batch.argtypes = [vp]
    L.geo_dist_to_boundary_batched.argtypes = [vp, dp, dp, dp, dp, dp, dp, i64, dp, ip, vp]
    L.geo_dist_to_boundary_batched_noalloc.argtypes = [ctypes.POINTER(vp), i32, ctypes.POINTER(geo_basket), i32,
                                                       dp, dp, dp, dp, dp, dp, i64, dp, ip, vp]
    L.geo_adjoint_workspace_size.argtypes = [vp, i64, ctypes.POINTER(ctypes.c_uint64)]
    L.geo_dist_to_boundary_adjoint.argtypes = [vp, dp, dp, dp, dp, dp, dp, i64, ip, dp, dp, dp, dp, dp, vp,
                                               ctypes.c_uint64, vp]
    L.geo_selftest_wait_timeout.argtypes = [vp, ctypes.c_uint32, vp]
    L.geo_debug_fail_alloc.argtypes = [i32]
    L.geo_status_string.argtypes = [ctypes.c_int]
    L.geo_status_string.restype = ctypes.c_char_p
    for name in EXPORTS:
        if name != "geo_status_string":
            getattr(L, name).restype = ctypes.c_int
    _lib = L
    return L


def geo_status_string(status: int) -> str:
    return load().geo_status_string(int(status)).decode()


def _check(st: int, what: str):
    if st != GEO_OK:
        raise GeoError(st, what)


def _stream(stream):
    import torch

    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(int(stream.cuda_stream) if hasattr(stream, "cuda_stream") else int(stream))


def _shape_struct(kind, params, rot=None, trans=None, pdata=None, keep=None) -> geo_placed_shape:
    """params: the solid's row; for a polycone either a spec with z, rmin,
    rmax, sphi, dphi, or a row (sphi, dphi, nz, offset, 0) into `pdata`.  The
    plane array is appended to `keep`, which the caller holds until the call
    that receives the struct returns."""
    s = geo_placed_shape()
    s.kind = int(kind)
    s.reserved = 0
    p = np.zeros(5)
    if int(kind) == GEO_PCON:
        if hasattr(params, "rmax"):
            planes = np.concatenate([np.asarray(params.z, float), np.asarray(params.rmin, float),
                                     np.asarray(params.rmax, float)])
            p[:3] = (params.sphi, params.dphi, len(params.z))
        else:
            nz, off = int(params[2]), int(params[3])
            planes = np.asarray(pdata, dtype=np.float64)[off: off + 3 * nz]
            p[:3] = (params[0], params[1], nz)
        planes = np.ascontiguousarray(planes, dtype=np.float64)
        if keep is None:
            raise ValueError("a polycone needs a keep list for its plane array")
        keep.append(planes)
        s.planes = planes.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    else:
        p[: len(params)] = params
    s.p[:] = [float(v) for v in p]
    s.rot[:] = [float(v) for v in (np.eye(3).reshape(9) if rot is None else np.asarray(rot).reshape(9))]
    s.trans[:] = [float(v) for v in (np.zeros(3) if trans is None else np.asarray(trans).reshape(3))]
    return s


class Volume:
    """Owns one geo_volume handle (device tables of a mother and its daughters)."""

    def __init__(self, handle, n_daughters: int):
        self.handle = handle
        self.n_daughters = n_daughters

    def close(self):
        if self.handle:
            load().geo_destroy_volume(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def _as_parameter_(self):
        return self.handle


def geo_build_volume(scene, voxelize: bool = False, grid=(0, 0, 0), stream=None) -> Volume:
    """Builds the device tables of `scene` (an object with mother_kind,
    mother_params, kinds, params, rot, trans -- see scenes.Scene)."""
    L = load()
    keep = []
    pdata = getattr(scene, "pdata", None)
    mother = _shape_struct(scene.mother_kind, scene.mother_params, pdata=pdata, keep=keep)
    nd = int(scene.n_daughters)
    arr = (geo_placed_shape * max(nd, 1))()
    for j in range(nd):
        arr[j] = _shape_struct(scene.kinds[j], scene.params[j], scene.rot[j], scene.trans[j], pdata=pdata, keep=keep)
    opts = geo_build_opts()
    opts.voxelize = 1 if voxelize else 0
    opts.grid[:] = [int(g) for g in grid]
    out = ctypes.c_void_p()
    _check(L.geo_build_volume(ctypes.byref(mother), arr, nd, ctypes.byref(opts), _stream(stream),
                              ctypes.byref(out)), "geo_build_volume")
    return Volume(out, nd)


def geo_destroy_volume(vol: Volume):
    vol.close()


def geo_volume_info(vol: Volume):
    nd, vx = ctypes.c_int32(), ctypes.c_int32()
    g = (ctypes.c_int32 * 3)()
    _check(load().geo_volume_info(vol.handle, ctypes.byref(nd), ctypes.byref(vx), ctypes.byref(g)),
           "geo_volume_info")
    return {"n_daughters": nd.value, "voxelized": bool(vx.value), "grid": tuple(g)}


def _dev(t, dtype, n, name):
    import torch

    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name}: expected a CUDA tensor")
    if t.dtype != dtype or not t.is_contiguous() or t.numel() != n:
        raise ValueError(f"{name}: expected contiguous {dtype} with {n} elements")
    return ctypes.c_void_p(t.data_ptr())


def geo_dist_to_boundary(vol: Volume, x, y, z, dx, dy, dz, mode: int = GEO_FP32_REFINE, step=None, hit=None,
                         bpoint=None, want_bpoint: bool = False, stream=None):
    """Fig. 1 navigator step for a basket of CUDA float64 tensors.  Returns
    (step, hit) or (step, hit, bpoint[3, n])."""
    import torch

    n = int(x.numel())
    f64 = torch.float64
    if step is None:
        step = torch.empty(n, dtype=f64, device=x.device)
    if hit is None:
        hit = torch.empty(n, dtype=torch.int32, device=x.device)
    if want_bpoint and bpoint is None:
        bpoint = torch.empty((3, n), dtype=f64, device=x.device)
    args = [_dev(a, f64, n, nm) for a, nm in ((x, "x"), (y, "y"), (z, "z"), (dx, "dx"), (dy, "dy"), (dz, "dz"))]
    bp = _dev(bpoint, f64, 3 * n, "bpoint") if bpoint is not None else ctypes.c_void_p(0)
    _check(load().geo_dist_to_boundary(vol.handle, *args, n, _dev(step, f64, n, "step"),
                                       _dev(hit, torch.int32, n, "hit"), bp, int(mode), _stream(stream)),
           "geo_dist_to_boundary")
    return (step, hit, bpoint) if bpoint is not None else (step, hit)


def geo_contains(vol: Volume, x, y, z, mode: int = GEO_FP32_REFINE, where=None, stream=None):
    """Navigator-level Contains: -2 outside the mother, -1 mother only, else
    the lowest-index daughter containing the point (same answer in both
    modes)."""
    import torch

    n = int(x.numel())
    if where is None:
        where = torch.empty(n, dtype=torch.int32, device=x.device)
    f64 = torch.float64
    _check(load().geo_contains(vol.handle, _dev(x, f64, n, "x"), _dev(y, f64, n, "y"), _dev(z, f64, n, "z"), n,
                               _dev(where, torch.int32, n, "where"), int(mode), _stream(stream)), "geo_contains")
    return where


def geo_safety(vol: Volume, x, y, z, mode: int = GEO_FP32_REFINE, safety=None, stream=None):
    """Navigator-level Safety: exact Euclidean in GEO_FP64 and GEO_FP32_REFINE
    (the same FP64 value), or the cheaper lower bound with
    GEO_SAFETY_ESTIMATE."""
    import torch

    n = int(x.numel())
    f64 = torch.float64
    if safety is None:
        safety = torch.empty(n, dtype=f64, device=x.device)
    _check(load().geo_safety(vol.handle, _dev(x, f64, n, "x"), _dev(y, f64, n, "y"), _dev(z, f64, n, "z"), n,
                             _dev(safety, f64, n, "safety"), int(mode), _stream(stream)), "geo_safety")
    return safety


GEO_Q_DIST_OUT, GEO_Q_DIST_IN, GEO_Q_SAFETY_OUT, GEO_Q_SAFETY_IN, GEO_Q_CONTAINS = range(5)


def geo_shape_query(kind, params, what, x, y, z, dx=None, dy=None, dz=None, rot=None, trans=None, out=None,
                    face=None, want_face=False, stream=None):
    """One solid's DistFromOutside / DistFromInside / safeties / Contains for a
    basket of CUDA float64 tensors (positions in the frame the solid is placed
    in).  Returns out, or (out, face) with want_face."""
    import torch

    n = int(x.numel())
    f64 = torch.float64
    if out is None:
        out = torch.empty(n, dtype=f64, device=x.device)
    if want_face and face is None:
        face = torch.empty(n, dtype=torch.int32, device=x.device)
    keep = []
    shape = _shape_struct(kind, params, rot, trans, keep=keep)
    dist = what in (GEO_Q_DIST_OUT, GEO_Q_DIST_IN)
    dirs = [_dev(a, f64, n, nm) if dist else ctypes.c_void_p(0) for a, nm in ((dx, "dx"), (dy, "dy"), (dz, "dz"))]
    _check(load().geo_shape_query(ctypes.byref(shape), int(what), _dev(x, f64, n, "x"), _dev(y, f64, n, "y"),
                                  _dev(z, f64, n, "z"), *dirs, n, _dev(out, f64, n, "out"),
                                  _dev(face, torch.int32, n, "face") if face is not None else ctypes.c_void_p(0),
                                  _stream(stream)), "geo_shape_query")
    return (out, face) if want_face else out


class World:
    """Owns one geo_world handle (a tree of logical volumes); keeps its
    volumes alive."""

    def __init__(self, handle, volumes, n_nodes: int, max_depth: int):
        self.handle = handle
        self.volumes = list(volumes)
        self.n_nodes = n_nodes
        self.max_depth = max_depth

    def close(self):
        if self.handle:
            load().geo_destroy_world(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def geo_build_world(volumes, child, root: int = 0, stream=None) -> World:
    """volumes: list of Volume (logical volumes); child: per volume, the
    volume index placed as each of its daughters (list of lists, or the
    concatenated int array); root: index of the top volume."""
    L = load()
    nv = len(volumes)
    handles = (ctypes.c_void_p * max(nv, 1))(*[v.handle for v in volumes])
    flat = np.concatenate([np.asarray(c, dtype=np.int32).reshape(-1) for c in child]) if len(child) and \
        not np.isscalar(child[0]) else np.asarray(child, dtype=np.int32)
    flat = np.ascontiguousarray(flat, dtype=np.int32)
    out = ctypes.c_void_p()
    _check(L.geo_build_world(handles, nv, flat.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), int(root),
                             _stream(stream), ctypes.byref(out)), "geo_build_world")
    nn, md = ctypes.c_int32(), ctypes.c_int32()
    _check(L.geo_world_info(out, ctypes.byref(nn), ctypes.byref(md)), "geo_world_info")
    return World(out, volumes, nn.value, md.value)


def geo_destroy_world(world: World):
    world.close()


def geo_world_info(world: World):
    nn, md = ctypes.c_int32(), ctypes.c_int32()
    _check(load().geo_world_info(world.handle, ctypes.byref(nn), ctypes.byref(md)), "geo_world_info")
    return nn.value, md.value


def geo_world_nodes(world: World) -> dict:
    """Node table (host numpy int32 arrays): lv, parent, slot, first."""
    n = world.n_nodes
    arrs = [np.empty(n, dtype=np.int32) for _ in range(4)]
    _check(load().geo_world_nodes(world.handle, *[a.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)) for a in arrs]),
           "geo_world_nodes")
    return dict(zip(("lv", "parent", "slot", "first"), arrs))


def geo_world_locate(world: World, x, y, z, node=None, stream=None):
    import torch

    n = int(x.numel())
    f64 = torch.float64
    if node is None:
        node = torch.empty(n, dtype=torch.int32, device=x.device)
    _check(load().geo_world_locate(world.handle, _dev(x, f64, n, "x"), _dev(y, f64, n, "y"), _dev(z, f64, n, "z"), n,
                                   _dev(node, torch.int32, n, "node"), _stream(stream)), "geo_world_locate")
    return node


def geo_world_step(world: World, x, y, z, dx, dy, dz, node, flag=None, mode: int = GEO_FP32_REFINE, step=None,
                   node_out=None, flag_out=None, stream=None):
    """One step of every track in its node, then relocation.  Returns
    (step, node_out, flag_out)."""
    import torch

    n = int(x.numel())
    f64 = torch.float64
    if step is None:
        step = torch.empty(n, dtype=f64, device=x.device)
    if node_out is None:
        node_out = torch.empty(n, dtype=torch.int32, device=x.device)
    if flag_out is None:
        flag_out = torch.empty(n, dtype=torch.int32, device=x.device)
    args = [_dev(a, f64, n, nm) for a, nm in ((x, "x"), (y, "y"), (z, "z"), (dx, "dx"), (dy, "dy"), (dz, "dz"))]
    _check(load().geo_world_step(world.handle, *args, n, _dev(node, torch.int32, n, "node"),
                                 _dev(flag, torch.int32, n, "flag") if flag is not None else ctypes.c_void_p(0),
                                 _dev(step, f64, n, "step"), _dev(node_out, torch.int32, n, "node_out"),
                                 _dev(flag_out, torch.int32, n, "flag_out"), int(mode), _stream(stream)),
           "geo_world_step")
    return step, node_out, flag_out


def geo_dist_to_boundary_host(vol: Volume, x, y, z, dx, dy, dz, mode: int = GEO_FP32_REFINE, step=None, hit=None,
                              chunk: int = 0, stream=None):
    """Host-memory variant: numpy float64 arrays or CPU tensors in, outputs
    filled (numpy arrays, or pinned tensors when the inputs are pinned
    tensors and no outputs are given); synchronises the stream.  With every
    array pinned the step runs on them in place; otherwise the library stages
    them through device buffers in chunks."""
    n = int(len(x))
    if step is None and hit is None and all(hasattr(a, "is_pinned") and a.is_pinned() for a in (x, y, z, dx, dy, dz)):
        import torch

        step = torch.empty(n, dtype=torch.float64, pin_memory=True)
        hit = torch.empty(n, dtype=torch.int32, pin_memory=True)

    def ptr(a):
        if hasattr(a, "data_ptr"):
            return ctypes.c_void_p(a.data_ptr())
        if a.dtype not in (np.float64, np.int32) or not a.flags["C_CONTIGUOUS"]:
            raise ValueError("host arrays must be contiguous float64 / int32")
        return ctypes.c_void_p(a.ctypes.data)

    if step is None:
        step = np.empty(n)
    if hit is None:
        hit = np.empty(n, dtype=np.int32)
    _check(load().geo_dist_to_boundary_host(vol.handle, *(ptr(a) for a in (x, y, z, dx, dy, dz)), n, ptr(step),
                                            ptr(hit), int(mode), int(chunk), _stream(stream)),
           "geo_dist_to_boundary_host")
    return step, hit


def geo_dist_to_boundary_stats(vol: Volume, x, y, z, dx, dy, dz, stream=None):
    """FP32+refine step that also returns the per-track count of FP64 solid
    evaluations.  Returns (step, hit, nref)."""
    import torch

    n = int(x.numel())
    f64 = torch.float64
    step = torch.empty(n, dtype=f64, device=x.device)
    hit = torch.empty(n, dtype=torch.int32, device=x.device)
    nref = torch.empty(n, dtype=torch.int32, device=x.device)
    args = [_dev(a, f64, n, nm) for a, nm in ((x, "x"), (y, "y"), (z, "z"), (dx, "dx"), (dy, "dy"), (dz, "dz"))]
    _check(load().geo_dist_to_boundary_stats(vol.handle, *args, n, _dev(step, f64, n, "step"),
                                             _dev(hit, torch.int32, n, "hit"), _dev(nref, torch.int32, n, "nref"),
                                             _stream(stream)), "geo_dist_to_boundary_stats")
    return step, hit, nref


def geo_check_device_status(vol: Volume, stream=None) -> int:
    """Reads and clears the volume's device error word; raises GeoError if set."""
    w = ctypes.c_uint32()
    st = load().geo_check_device_status(vol.handle, ctypes.byref(w), _stream(stream))
    if st not in (GEO_OK, 5):
        _check(st, "geo_check_device_status")
    if st == 5:
        raise GeoError(st, f"device status word 0x{w.value:x}")
    return w.value


def geo_selftest_wait_timeout(vol: Volume, polls: int = 256, stream=None):
    """Runs the failure path of a bounded wait (a barrier nobody arrives at);
    the volume's status word then holds bit 4 (see geo.h)."""
    _check(load().geo_selftest_wait_timeout(vol.handle, int(polls), _stream(stream)), "geo_selftest_wait_timeout")


def geo_debug_fail_alloc(nth: int):
    """Host-side fault injection: the nth allocation of the library from now
    on fails as out of memory (0: off).  See geo.h."""
    _check(load().geo_debug_fail_alloc(int(nth)), "geo_debug_fail_alloc")


def geo_probe_pipe(what: int, iters: int = 1 << 16, blocks: int = 0, stream=None) -> float:
    """Operations per second of one arithmetic operation (see geo.h)."""
    import torch

    if blocks <= 0:
        blocks = torch.cuda.get_device_properties(0).multi_processor_count * 8
    scratch = torch.empty(256, dtype=torch.float64, device="cuda")
    r = ctypes.c_double()
    _check(load().geo_probe_pipe(int(what), int(iters), int(blocks), ctypes.c_void_p(scratch.data_ptr()),
                                 _stream(stream), ctypes.byref(r)), "geo_probe_pipe")
    return r.value


class Batch:
    """Owns one geo_batch handle; keeps its volumes alive."""

    def __init__(self, handle, volumes, ntracks_needed):
        self.handle = handle
        self.volumes = list(volumes)
        self.ntracks_needed = ntracks_needed

    def close(self):
        if self.handle:
            load().geo_destroy_batch(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def geo_build_batch(volumes, baskets, tile_order: int = 0, blocks_per_sm: int = 0, tile_tracks: int = 0,
                    stream=None) -> Batch:
    """volumes: list of Volume; baskets: (volume index, offset, count) rows;
    tile_tracks: 0 / GEO_TILE_TRACKS (384) or 256 (see geo.h)."""
    L = load()
    nv = len(volumes)
    handles = (ctypes.c_void_p * max(nv, 1))(*[v.handle for v in volumes])
    rows = np.asarray(baskets, dtype=np.int64).reshape(-1, 3)
    arr = (geo_basket * max(len(rows), 1))()
    for k, (v, off, cnt) in enumerate(rows):
        arr[k].volume, arr[k].reserved, arr[k].offset, arr[k].count = int(v), 0, int(off), int(cnt)
    opts = geo_batch_opts()
    opts.tile_order, opts.blocks_per_sm, opts.tile_tracks = int(tile_order), int(blocks_per_sm), int(tile_tracks)
    out = ctypes.c_void_p()
    _check(L.geo_build_batch(handles, nv, arr, len(rows), ctypes.byref(opts), _stream(stream), ctypes.byref(out)),
           "geo_build_batch")
    need = int((rows[:, 1] + rows[:, 2]).max()) if len(rows) else 0
    return Batch(out, volumes, need)


def geo_destroy_batch(batch: Batch):
    batch.close()


def geo_dist_to_boundary_batched(batch: Batch, x, y, z, dx, dy, dz, step=None, hit=None, stream=None):
    """One persistent launch over every basket of the batch (FP32+refine)."""
    import torch

    n = int(x.numel())
    f64 = torch.float64
    if step is None:
        step = torch.empty(n, dtype=f64, device=x.device)
    if hit is None:
        hit = torch.empty(n, dtype=torch.int32, device=x.device)
    args = [_dev(a, f64, n, nm) for a, nm in ((x, "x"), (y, "y"), (z, "z"), (dx, "dx"), (dy, "dy"), (dz, "dz"))]
    _check(load().geo_dist_to_boundary_batched(batch.handle, *args, n, _dev(step, f64, n, "step"),
                                               _dev(hit, torch.int32, n, "hit"), _stream(stream)),
           "geo_dist_to_boundary_batched")
    return step, hit


def geo_dist_to_boundary_batched_noalloc(volumes, baskets, x, y, z, dx, dy, dz, step, hit, stream=None):
    """Batched step without any device allocation by the call (the library's
    fixed scratch array is used instead): for callers that cannot let a
    library allocate while they run.  step / hit must be preallocated CUDA
    tensors.  Calls sharing the scratch must not overlap on the GPU."""
    import torch

    n = int(x.numel())
    f64 = torch.float64
    nv = len(volumes)
    handles = (ctypes.c_void_p * max(nv, 1))(*[v.handle for v in volumes])
    rows = np.asarray(baskets, dtype=np.int64).reshape(-1, 3)
    arr = (geo_basket * max(len(rows), 1))()
    for k, (v, off, cnt) in enumerate(rows):
        arr[k].volume, arr[k].reserved, arr[k].offset, arr[k].count = int(v), 0, int(off), int(cnt)
    args = [_dev(a, f64, n, nm) for a, nm in ((x, "x"), (y, "y"), (z, "z"), (dx, "dx"), (dy, "dy"), (dz, "dz"))]
    _check(load().geo_dist_to_boundary_batched_noalloc(handles, nv, arr, len(rows), *args, n,
                                                       _dev(step, f64, n, "step"), _dev(hit, torch.int32, n, "hit"),
                                                       _stream(stream)), "geo_dist_to_boundary_batched_noalloc")
    return step, hit


def geo_adjoint_workspace_size(vol: Volume, n: int) -> int:
    b = ctypes.c_uint64()
    _check(load().geo_adjoint_workspace_size(vol.handle, int(n), ctypes.byref(b)), "geo_adjoint_workspace_size")
    return int(b.value)


def geo_dist_to_boundary_adjoint(vol: Volume, x, y, z, dx, dy, dz, hit, grad_step, want_geometry: bool = True,
                                 stream=None):
    """Gradients of sum(grad_step * step): returns grad_p (3, n), grad_d (3, n)
    and, when want_geometry, grad_trans (nd, 3) and grad_params (nd + 1, 5)
    (the mother's parameters last)."""
    import torch

    n = int(x.numel())
    f64 = torch.float64
    nd = vol.n_daughters
    gp = torch.empty((3, n), dtype=f64, device=x.device)
    gd = torch.empty((3, n), dtype=f64, device=x.device)
    gt = torch.zeros((max(nd, 1), 3), dtype=f64, device=x.device) if want_geometry else None
    gprm = torch.zeros((nd + 1, 5), dtype=f64, device=x.device) if want_geometry else None
    ws = torch.empty(max(geo_adjoint_workspace_size(vol, n), 8) // 8 + 1, dtype=f64, device=x.device)
    args = [_dev(a, f64, n, nm) for a, nm in ((x, "x"), (y, "y"), (z, "z"), (dx, "dx"), (dy, "dy"), (dz, "dz"))]
    _check(load().geo_dist_to_boundary_adjoint(
        vol.handle, *args, n, _dev(hit, torch.int32, n, "hit"), _dev(grad_step, f64, n, "grad_step"),
        _dev(gp, f64, 3 * n, "grad_p"), _dev(gd, f64, 3 * n, "grad_d"),
        ctypes.c_void_p(gt.data_ptr()) if gt is not None else ctypes.c_void_p(0),
        ctypes.c_void_p(gprm.data_ptr()) if gprm is not None else ctypes.c_void_p(0),
        ctypes.c_void_p(ws.data_ptr()), ctypes.c_uint64(ws.numel() * 8), _stream(stream)),
        "geo_dist_to_boundary_adjoint")
    if not want_geometry:
        return gp, gd
    return gp, gd, gt[:nd], gprm
