"""Contains and Safety (Sec. 3.1) on the GPU: the FP32-filtered mode against
the plain FP64 mode (same answers, bit for bit, on every point) and both
against the oracle.

Points: uniform in the mother (daughters included), points on the surfaces
(oracle boundary points p + s d of random tracks: every kind of face, the
mother's included) and those points moved by +-1e-7 mm and +-1e-12 mm along
the track, points in the band between the mother's deflated and inflated FP32
copies, and non-finite points.  Scenes cover the staged FP32 table (up to 768
daughters) and the global-memory one (1000 daughters).
"""
import numpy as np
import pytest

from paper_1312_0816_gb300 import scenes

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

STEP_TOL = 1e-9


@pytest.fixture(scope="module")
def g():
    import paper_1312_0816_gb300 as pkg

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    pkg.load()
    return pkg


def scene_list():
    return [scenes.toy40(1), scenes.toy8(1), scenes.box4(0), scenes.diff3(), scenes.grid512(5),
            scenes.cell_volume(11, 200, False), scenes.cell_volume(12, 1000, True), scenes.seg4(), scenes.pcon4(),
            scenes.pconm()]


def hard_points(orc, sc, n, seed):
    rng = np.random.default_rng(seed)
    tr = scenes.sample_tracks(sc, n, seed)
    ref = orc.navigate(sc, tr, nthreads=8)
    s = ref["step"]
    pts = [np.stack([tr.x, tr.y, tr.z], 1)]
    d = np.stack([tr.dx, tr.dy, tr.dz], 1)
    on = pts[0] + s[:, None] * d
    pts.append(on)
    for eps in (1e-7, -1e-7, 1e-12, -1e-12):
        pts.append(on + eps * d)
    # points just inside the mother's boundary (the FP32 band of the mother)
    m = ref["hit"] == -1
    for eps in (1e-4, 1e-6, 1e-9):
        pts.append(on[m] - eps * d[m])
    p = np.concatenate(pts)
    p = p[rng.permutation(p.shape[0])]
    bad = np.array([[np.nan, 0, 0], [0, np.inf, 0], [0, 0, -np.inf], [1e300, 0, 0]])
    p = np.concatenate([p, bad])
    z = np.zeros(p.shape[0])
    return scenes.Tracks(p[:, 0].copy(), p[:, 1].copy(), p[:, 2].copy(), z + 1.0, z, z)


def dev3(tr):
    return [torch.from_numpy(np.ascontiguousarray(f)).cuda() for f in (tr.x, tr.y, tr.z)]


@pytest.mark.parametrize("idx", range(10))
def test_modes_agree_and_match_oracle(g, orc, idx):
    sc = scene_list()[idx]
    vol = g.geo_build_volume(sc)
    for tr in (scenes.sample_tracks(sc, 50000, 20 + idx, exclusive=False), hard_points(orc, sc, 20000, 30 + idx)):
        x = dev3(tr)
        w = [g.geo_contains(vol, *x, mode=m).cpu().numpy() for m in (0, 1)]
        s = [g.geo_safety(vol, *x, mode=m).cpu().numpy() for m in (0, 1)]
        assert np.array_equal(w[0], w[1]), sc.name
        assert np.array_equal(s[0], s[1], equal_nan=True), sc.name
        want_w = orc.contains(sc, tr, nthreads=8)
        want_s = orc.safety(sc, tr, nthreads=8)
        finite = np.isfinite(tr.x) & np.isfinite(tr.y) & np.isfinite(tr.z)
        assert np.all(w[1][~finite] == -2) and np.all(s[1][~finite] == 0.0)
        # Contains is exact away from surfaces: points whose oracle safety is
        # below 1e-9 mm may differ (surface band)
        band = (want_s < STEP_TOL) | ~finite
        assert np.array_equal(w[1][~band], want_w[~band]), sc.name
        assert np.max(np.abs(s[1] - want_s)[finite]) <= STEP_TOL, sc.name
    assert g.geo_check_device_status(vol) == 0
    vol.close()


def test_empty_and_single(g):
    sc = scenes.toy40(1)
    vol = g.geo_build_volume(sc)
    e = torch.empty(0, dtype=torch.float64, device="cuda")
    assert g.geo_contains(vol, e, e, e, mode=1).numel() == 0
    assert g.geo_safety(vol, e, e, e, mode=1).numel() == 0
    one = torch.tensor([0.0], dtype=torch.float64, device="cuda")
    # on the axis at the centre: inside the innermost shell's hole, mother only
    assert int(g.geo_contains(vol, one, one, one, mode=1).item()) == -1
    assert float(g.geo_safety(vol, one, one, one, mode=1).item()) == 40.0
    vol.close()


def test_mother_only_volume(g, orc):
    sc = scenes.Scene("empty", scenes.TUBE, np.array([10.0, 100.0, 50.0, 0, 0]), np.zeros(0, np.int32),
                      np.zeros((0, 5)), np.zeros((0, 9)), np.zeros((0, 3)))
    vol = g.geo_build_volume(sc)
    tr = scenes.sample_tracks(sc, 10000, 5)
    x = dev3(tr)
    for m in (0, 1):
        assert np.array_equal(g.geo_contains(vol, *x, mode=m).cpu().numpy(), orc.contains(sc, tr))
        got = g.geo_safety(vol, *x, mode=m).cpu().numpy()
        assert np.max(np.abs(got - orc.safety(sc, tr))) <= STEP_TOL
    vol.close()


EPS32 = 2.0 ** -24


def _radius_and_slope(kind, row, pcon_planes=None):
    """Bounding radius of the solid's FP32 copy and its largest radius slope
    squared (a segment or polycone is copied as its enclosing tube)."""
    if kind == scenes.BOX:
        return float(np.sqrt(np.sum(np.asarray(row[:3]) ** 2))), 0.0
    if kind in (scenes.TUBE, scenes.TUBS):
        return float(np.hypot(row[1], row[2])), 0.0
    if kind == scenes.PCON:
        z, _, rx = pcon_planes
        return float(np.hypot(rx.max(), 0.5 * (z[-1] - z[0]))), 0.0
    dz = row[0]
    b2 = max(((row[4] - row[2]) / (2 * dz)) ** 2, ((row[3] - row[1]) / (2 * dz)) ** 2)
    return float(np.hypot(max(row[2], row[4]), dz)), b2


def inflation_bound(sc):
    """An upper bound of the FP32 inflation of the volume's solids, from the
    builder's rule: eps32 (48 S + 16 br) for the rounding of positions and of
    the shape arithmetic, plus a discriminant term that its radius floor
    bounds by 32 sqrt(eps32) br (1 + b^2); S is the mother's extent."""
    if sc.mother_kind == scenes.PCON:
        z, _, rx = sc.planes_of(sc.mother_params)
        S = float(np.sqrt(rx * rx + z * z).max())
    else:
        S, _ = _radius_and_slope(sc.mother_kind, sc.mother_params)
    worst = 0.0
    solids = [(sc.mother_kind, sc.mother_params)] + [(int(k), sc.params[j]) for j, k in enumerate(sc.kinds)]
    for kind, row in solids:
        br, b2 = _radius_and_slope(kind, row, sc.planes_of(row) if kind == scenes.PCON else None)
        d = EPS32 * (48 * S + 16 * br)
        if kind != scenes.BOX:
            d += 32 * np.sqrt(EPS32) * br * (1 + b2)
        worst = max(worst, d)
    return worst


@pytest.mark.parametrize("idx", range(10))
def test_safety_estimate(g, orc, idx):
    """GEO_SAFETY_ESTIMATE: never above the exact safety nor above the defined
    bound (the oracle's estimate), and below that bound by at most twice the
    FP32 inflation plus a relative 2^-16; 0 for non-finite points."""
    sc = scene_list()[idx]
    vol = g.geo_build_volume(sc)
    tol_abs = 2.0 * inflation_bound(sc)
    uniform = scenes.sample_tracks(sc, 50000, 20 + idx, exclusive=False)
    for tr in (uniform, hard_points(orc, sc, 20000, 30 + idx)):
        est = g.geo_safety(vol, *dev3(tr), mode=2).cpu().numpy()
        want = orc.safety_estimate(sc, tr, nthreads=8)
        exact = orc.safety(sc, tr, nthreads=8)
        finite = np.isfinite(tr.x) & np.isfinite(tr.y) & np.isfinite(tr.z)
        assert np.all(est[~finite] == 0.0)
        assert np.all(est >= 0.0)
        assert np.all(est <= exact + 1e-12 * (1.0 + exact)), sc.name
        assert np.all(est <= want + 1e-12 * (1.0 + want)), sc.name
        assert np.all(est >= want - tol_abs - 2.0 ** -16 * want), (sc.name, float(np.max(want - est)), tol_abs)
        if tr is uniform and sc.mother_kind not in (scenes.TUBS, scenes.PCON):
            pos = exact > 0
            assert np.mean(est[pos] / exact[pos]) > 0.9, sc.name   # a useful bound, not just a valid one
    vol.close()
