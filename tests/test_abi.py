"""CPU-only checks of the C ABI: the library builds, loads, exports every
function include/geo.h declares, and rejects invalid arguments on the host
before touching the GPU."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_1312_0816_gb300 import geonav
from paper_1312_0816_gb300.geonav import geo_placed_shape

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared():
    src = open(os.path.join(ROOT, "include", "geo.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(geo_[a-z0-9_]+)\s*\(", src)))


def test_library_exports_every_declared_symbol():
    L = geonav.load()
    names = declared()
    assert "geo_dist_to_boundary" in names and "geo_build_volume" in names
    for name in names:
        assert hasattr(L, name), name
    # and the binding wraps each of them under the same name
    for name in names:
        assert hasattr(geonav, name), name


def test_binding_constants_match_the_header():
    """Every #define and enum constant of include/geo.h has the same value in
    the binding."""
    src = open(os.path.join(ROOT, "include", "geo.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    consts = {k: int(v) for k, v in re.findall(r"#define\s+(GEO_[A-Z0-9_]+)\s+(\d+)", src)}
    for body in re.findall(r"typedef enum\s*\{(.*?)\}", src, flags=re.S):
        consts.update({k: int(v) for k, v in re.findall(r"(GEO_[A-Z0-9_]+)\s*=\s*(\d+)", body)})
    assert {"GEO_MAX_PLANES", "GEO_TILE_TRACKS", "GEO_PCON", "GEO_SAFETY_ESTIMATE"} <= set(consts)
    for k, v in consts.items():
        if k.startswith("GEO_ERR_") or k == "GEO_OK":
            continue
        assert getattr(geonav, k) == v, k


def test_status_strings():
    for s in range(7):
        assert geonav.geo_status_string(s)
    assert geonav.geo_status_string(99) == "unknown status"


def _shape(kind, p, rot=None, trans=None):
    return geonav._shape_struct(kind, p, rot, trans)


def _build(mother, daughters):
    L = geonav.load()
    arr = (geo_placed_shape * max(1, len(daughters)))(*daughters)
    out = ctypes.c_void_p(123)
    st = L.geo_build_volume(ctypes.byref(mother), arr, len(daughters), None, None, ctypes.byref(out))
    return st, out


@pytest.mark.parametrize("mother,daughter,status", [
    ((0, (100, 100, 100)), (5, (1, 1, 1)), 1),                      # unknown kind
    ((0, (100, 100, 100)), (3, (0, 10, 5, 0, 0)), 2),               # tube segment of no angle
    ((0, (100, 100, 100)), (3, (0, 10, 5, 0, 7)), 2),               # tube segment beyond a whole turn
    ((0, (100, 100, 100)), (3, (8, 6, 5, 0, 1)), 2),                # tube segment rmin > rmax
    ((0, (100, 100, 100)), (1, (20, 10, 5)), 2),                    # rmin > rmax
    ((0, (100, 100, 100)), (1, (0, 10, 0)), 2),                     # dz = 0
    ((0, (100, 100, 100)), (2, (5, 3, 2, 0, 4)), 2),                # cone rmin1 > rmax1
    ((0, (100, 100, 100)), (2, (5, 0, 0, 0, 0)), 2),                # cone without radius
    ((0, (100, 100, 100)), (0, (1, float("nan"), 1)), 2),           # NaN parameter
    ((0, (100, -1, 100)), (0, (1, 1, 1)), 2),                       # bad mother
])
def test_build_rejects_bad_shapes(mother, daughter, status):
    st, out = _build(_shape(*mother), [_shape(*daughter)])
    assert st == status
    assert out.value is None


def test_build_rejects_non_orthonormal_rotation():
    rot = np.eye(3)
    rot[0, 1] = 1e-9
    st, out = _build(_shape(0, (100, 100, 100)), [_shape(0, (1, 1, 1), rot)])
    assert st == 2
    refl = np.diag([1.0, 1.0, -1.0])   # orthonormal but det = -1
    st, _ = _build(_shape(0, (100, 100, 100)), [_shape(0, (1, 1, 1), refl)])
    assert st == 2


def test_build_rejects_placed_mother():
    st, _ = _build(_shape(0, (100, 100, 100), None, (1.0, 0, 0)), [])
    assert st == 1


def test_null_arguments():
    L = geonav.load()
    assert L.geo_build_volume(None, None, 0, None, None, None) == 1
    m = _shape(0, (1, 1, 1))
    out = ctypes.c_void_p()
    assert L.geo_build_volume(ctypes.byref(m), None, 3, None, None, ctypes.byref(out)) == 1
    assert L.geo_dist_to_boundary(None, None, None, None, None, None, None, 0, None, None, None, 0, None) == 1
    assert L.geo_contains(None, None, None, None, 0, None, 0, None) == 1
    assert L.geo_safety(None, None, None, None, 0, None, 0, None) == 1
    assert L.geo_destroy_volume(None) == 0


def test_shape_query_validation():
    """Rejected before any device work: null shape, bad kind or parameters,
    unknown query, negative n; n == 0 with a valid solid is a no-op."""
    L = geonav.load()
    assert L.geo_shape_query(None, 0, None, None, None, None, None, None, 0, None, None, None) == 1
    good = _shape(1, (5, 10, 20))
    assert L.geo_shape_query(ctypes.byref(good), 0, None, None, None, None, None, None, 0, None, None, None) == 0
    assert L.geo_shape_query(ctypes.byref(good), 5, None, None, None, None, None, None, 0, None, None, None) == 1
    assert L.geo_shape_query(ctypes.byref(good), -1, None, None, None, None, None, None, 0, None, None, None) == 1
    assert L.geo_shape_query(ctypes.byref(good), 0, None, None, None, None, None, None, -1, None, None, None) == 1
    bad = _shape(1, (10, 5, 20))   # rmin > rmax
    assert L.geo_shape_query(ctypes.byref(bad), 0, None, None, None, None, None, None, 0, None, None, None) == 2
    kind = _shape(7, (1, 1, 1))
    assert L.geo_shape_query(ctypes.byref(kind), 0, None, None, None, None, None, None, 0, None, None, None) == 1


_KEEP = []


def _pcon(z, rmin, rmax, sphi=0.0, dphi=2 * np.pi, **over):
    from paper_1312_0816_gb300.scenes import Pcon

    s = geonav._shape_struct(4, Pcon(tuple(z), tuple(rmin), tuple(rmax), sphi, dphi), keep=_KEEP)
    for k, v in over.items():
        if k == "planes":
            s.planes = v
        else:
            s.p[int(k[1:])] = v
    return s


@pytest.mark.parametrize("shape,status", [
    (lambda: _pcon((-1, 0, 2), (0, 1, 0), (3, 4, 2)), 0),
    (lambda: _pcon((-1, 2), (0, 0), (3, 3), 0.5, 1.0), 0),                     # a cone segment
    (lambda: _pcon((-1, 2), (0, 0), (3, 3), planes=None), 1),                   # no plane table
    (lambda: _pcon((-1, 2), (0, 0), (3, 3), p2=1.0), 1),                        # one plane
    (lambda: _pcon((-1, 2), (0, 0), (3, 3), p2=2.5), 1),                        # not a count
    (lambda: _pcon(range(33), (0,) * 33, (1,) * 33), 1),                       # too many planes
    (lambda: _pcon((-1, -1, 2), (0, 0, 0), (3, 3, 3)), 2),                      # z not increasing
    (lambda: _pcon((-1, 0, 2), (0, 5, 0), (3, 4, 2)), 2),                       # rmin > rmax
    (lambda: _pcon((-1, 0, 2), (0, 0, 0), (0, 0, 2)), 2),                       # a section of no radius
    (lambda: _pcon((-1, 2), (0, 0), (3, 3), 0.0, 0.0), 2),                      # no angle
    (lambda: _pcon((-1, 2), (0, 0), (3, 3), 0.0, 7.0), 2),                      # beyond a whole turn
    (lambda: _pcon((-1, 2), (0, 0), (3, 3), p3=1.0), 2),                        # p[3] must be 0
    (lambda: _pcon((-1, 2), (0, float("nan")), (3, 3)), 2),                     # NaN radius
])
def test_polycone_validation(shape, status):
    """The polycone's rules (include/geo.h), checked before any device work."""
    L = geonav.load()
    s = shape()
    assert L.geo_shape_query(ctypes.byref(s), 0, None, None, None, None, None, None, 0, None, None, None) == status


def test_allocation_failure_returns_oom_on_the_host():
    """Host-side fault injection (geo_debug_fail_alloc): the library's first
    allocation of a build fails as if memory had run out, and the build
    returns GEO_ERR_OOM before it touches the GPU; with the hook off the same
    call goes on (here, without a GPU, to the device query)."""
    L = geonav.load()
    mother = _shape(0, (100, 100, 100))
    daughter = _shape(0, (10, 10, 10))
    assert L.geo_debug_fail_alloc(-1) == 1
    assert L.geo_debug_fail_alloc(1) == 0
    try:
        st, out = _build(mother, [daughter])
        assert st == 3 and out.value is None          # GEO_ERR_OOM, no handle
    finally:
        assert L.geo_debug_fail_alloc(0) == 0
    st, out = _build(mother, [daughter])
    assert st != 3


def test_selftest_rejects_bad_arguments():
    L = geonav.load()
    assert L.geo_selftest_wait_timeout(None, 16, None) == 1
