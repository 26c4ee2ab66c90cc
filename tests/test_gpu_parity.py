"""Parity of the CUDA navigator (through the C ABI) with the CPU oracle.

Bar, on every track: the step within max(1e-9 mm, err) of the oracle's, err
the oracle's a-priori FP64 error bound (pinned against exact crossings in
test_oracle_errbound.py; it exceeds 1e-9 mm only for ill-conditioned hits:
grazing incidence, near-tangent roots, far-away small solids), and the hit
index bit-exact except in the tie band (second-smallest oracle candidate
within that tolerance of the winner).  The share of conditioning-banded
tracks is capped on random rays.  The FP32+refine mode must equal the plain
FP64 mode bit for bit on every track.
"""
import math

import numpy as np
import pytest

from helpers import golden, expr, scene_from_spec, tracks_from, check_steps, STEP_TOL
from paper_1312_0816_gb300 import scenes

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def g():
    import paper_1312_0816_gb300 as pkg

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    pkg.load()
    return pkg


_vols = {}


def vol(g, sc):
    key = (sc.name, id(sc))
    if key not in _vols:
        _vols[key] = (sc, g.geo_build_volume(sc))
    return _vols[key][1]


def dev(tr):
    return [torch.from_numpy(np.ascontiguousarray(f)).cuda() for f in tr.fields()]


def run_nav(g, sc, tr, mode, bpoint=False):
    out = g.geo_dist_to_boundary(vol(g, sc), *dev(tr), mode=mode, want_bpoint=bpoint)
    torch.cuda.synchronize()
    return [o.cpu().numpy() for o in out]


def compare(ref, step, hit, tracks, sc, orc, max_banded=1e-3, max_graze=0.0):
    """Every track checked (helpers.check_steps); a track whose answer only
    FP64 rounding decides must be the oracle's for a start point moved by
    1e-9 mm, and their share is capped.  Returns the band counts."""
    st = check_steps(ref, step, hit, tracks, max_banded, orc, sc)
    assert st["rounding_decided"] <= max_graze * max(st["n"], 1), st
    return st


SCENES = {
    "box4": lambda: scenes.box4(0),
    "toy40": lambda: scenes.toy40(1),
    "toy8": lambda: scenes.toy8(1),
    "diff3": lambda: scenes.diff3(),
    "grid512": lambda: scenes.grid512(5),
    "seg4": lambda: scenes.seg4(),
    "pcon4": lambda: scenes.pcon4(),
    "pconm": lambda: scenes.pconm(),
}
_scene_cache = {}


def scene(name):
    if name not in _scene_cache:
        _scene_cache[name] = SCENES[name]()
    return _scene_cache[name]


@pytest.mark.parametrize("mode", [0, 1])
def test_box4_basket_1024(g, orc, mode):
    """The 1024-track basket in a box mother with four boxes (seed 0)."""
    sc = scene("box4")
    tr = scenes.sample_tracks(sc, 1024, 0)
    ref = orc.navigate(sc, tr, nthreads=8)
    step, hit = run_nav(g, sc, tr, mode)
    compare(ref, step, hit, tr, sc, orc)


@pytest.mark.parametrize("name,n", [("toy40", 65536 + 77), ("toy8", 30011), ("diff3", 30011),
                                    ("grid512", 8191), ("pcon4", 30011), ("pconm", 30011)])
@pytest.mark.parametrize("mode", [0, 1])
def test_scene_parity(g, orc, name, n, mode):
    """Several tiles of tracks (GEO_TILE_TRACKS, and the plain kernel's blocks of
    256) and a ragged tail."""
    sc = scene(name)
    tr = scenes.sample_tracks(sc, n, 101)
    ref = orc.navigate(sc, tr, nthreads=8)
    step, hit = run_nav(g, sc, tr, mode)
    compare(ref, step, hit, tr, sc, orc, max_graze=1e-4)


@pytest.mark.parametrize("name", list(SCENES))
def test_refine_equals_fp64_bitwise(g, name):
    """GEO_FP32_REFINE returns exactly the plain FP64 answers (random and
    adversarial grazing / edge / corner rays)."""
    sc = scene(name)
    for tr in (scenes.sample_tracks(sc, 50000, 7), scenes.adversarial_tracks(sc, 20000, 8)):
        s0, h0, b0 = run_nav(g, sc, tr, 0, bpoint=True)
        s1, h1, b1 = run_nav(g, sc, tr, 1, bpoint=True)
        assert np.array_equal(h0, h1)
        assert np.array_equal(s0.view(np.int64), s1.view(np.int64))
        assert np.array_equal(b0.view(np.int64), b1.view(np.int64))


@pytest.mark.parametrize("n", [5000, 200003])
def test_refine_fallback_to_the_full_loop(g, orc, n):
    """Five identical overlapping boxes (and one box apart): the entering
    distances of the five tie bit for bit, so their FP32 bounds tie too and
    the candidate list (two entries) has to evict one whose bound equals the
    best; those tracks take the full FP64 loop.  The answers are the oracle's
    (a tie goes to the lowest index) and the plain FP64 kernel's bits, in both
    block configurations of the filter kernel."""
    eye = np.eye(3).reshape(9)
    box = (0, (20.0, 30.0, 40.0), eye, (0.0, 0.0, 0.0))
    other = (0, (10.0, 10.0, 10.0), eye, (0.0, 150.0, 0.0))
    sc = scene_from_spec((0, (400.0, 400.0, 400.0)), [other, box, box, box, box, box], name="ties")
    rng = np.random.default_rng(23)
    side = np.where(rng.random(n) < 0.5, -1.0, 1.0)
    p = np.stack([60.0 * side, rng.uniform(-25.0, 25.0, n), rng.uniform(-35.0, 35.0, n)], axis=1)
    d = rng.normal(scale=0.3, size=(n, 3))
    d[:, 0] = -side
    d /= np.linalg.norm(d, axis=1)[:, None]
    tr = tracks_from(p, d)
    ref = orc.navigate(sc, tr, nthreads=8)
    s0, h0 = run_nav(g, sc, tr, 0)
    s1, h1 = run_nav(g, sc, tr, 1)
    assert np.array_equal(h0, h1) and np.array_equal(s0.view(np.int64), s1.view(np.int64))
    assert np.array_equal(h1, ref["hit"])
    assert np.max(np.abs(s1 - ref["step"])) <= STEP_TOL
    assert np.mean(h1 == 1) > 0.5 and not np.any(h1 >= 2)   # every box hit goes to the first copy
    _, _, nref = g.geo_dist_to_boundary_stats(vol(g, sc), *dev(tr))
    assert np.mean(nref.cpu().numpy() >= 1000) > 0.5


@pytest.mark.parametrize("name", list(SCENES))
def test_refine_block_configurations(g, name):
    """Both block configurations of the filter kernel -- 8 + 4 warps with
    tiles of 256 tracks while a basket has at most two tiles for each of two
    blocks per SM, 12 + 4 warps with tiles of GEO_TILE_TRACKS beyond -- return
    the plain FP64 bits, on either side of the switch and with a ragged tail."""
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    edge = 4 * sms * 256
    sc = scene(name)
    base = scenes.sample_tracks(sc, edge + 3 * g.GEO_TILE_TRACKS + 17, 21)
    for n in (edge, edge + 1, base.n):
        tr = scenes.Tracks(*(f[:n] for f in base.fields()))
        s0, h0 = run_nav(g, sc, tr, 0)
        s1, h1 = run_nav(g, sc, tr, 1)
        assert np.array_equal(h0, h1), n
        assert np.array_equal(s0.view(np.int64), s1.view(np.int64)), n


@pytest.mark.parametrize("name", ["box4", "toy40", "diff3", "grid512", "seg4", "pcon4", "pconm"])
def test_adversarial_parity(g, orc, name):
    sc = scene(name)
    tr = scenes.adversarial_tracks(sc, 20000, 9)
    ref = orc.navigate(sc, tr, nthreads=8)
    step, hit = run_nav(g, sc, tr, 1)
    # these rays are aimed at edges, rims and faces at grazing incidence, so a
    # large share is ill-conditioned by construction: every one of them is
    # still checked, at its own bound
    st = compare(ref, step, hit, tr, sc, orc, max_banded=None, max_graze=0.01)
    assert st["n"] == tr.n and st["cond_banded"] > 0


@pytest.mark.parametrize("name", ["toy8", "box4", "diff3", "seg4", "pcon4", "pconm"])
def test_small_basket_warp_path(g, name):
    """Baskets of at most 8 tracks per SM in volumes of at most 32 daughters
    take the warp-per-track kernel (lanes over daughters, shuffle minimum over
    (step, index)): the same bits as the thread-per-track kernels give the
    same tracks inside a large basket, in both modes."""
    sc = scene(name)
    tr = scenes.sample_tracks(sc, 40000, 31)
    adv = scenes.adversarial_tracks(sc, 3000, 32)
    for big in (tr, adv):
        n_small = 1000
        small = scenes.Tracks(*(f[:n_small].copy() for f in big.fields()))
        for mode in (0, 1):
            s_big, h_big, b_big = run_nav(g, sc, big, mode, bpoint=True) if big.n > 20000 else (None, None, None)
            if s_big is None:
                # pad the adversarial rays into a large basket with random ones
                joined = scenes.Tracks(*(np.concatenate([a, b]) for a, b in zip(big.fields(), tr.fields())))
                s_big, h_big, b_big = run_nav(g, sc, joined, mode, bpoint=True)
            s_sm, h_sm, b_sm = run_nav(g, sc, small, mode, bpoint=True)
            assert np.array_equal(s_sm.view(np.int64), s_big[:n_small].view(np.int64)), (name, mode)
            assert np.array_equal(h_sm, h_big[:n_small]), (name, mode)
            assert np.array_equal(b_sm.view(np.int64), b_big[:, :n_small].view(np.int64)), (name, mode)


@pytest.mark.parametrize("case", golden("closed_forms.json")["nav_cases"], ids=lambda c: c["why"][:40])
@pytest.mark.parametrize("mode", [0, 1])
def test_golden_navigator_cases(g, case, mode):
    sc = scene_from_spec(case["mother"], case["daughters"], name="golden" + case["why"][:20])
    tr = tracks_from(case["p"], case["d"])
    step, hit = run_nav(g, sc, tr, mode)
    want = expr(case["step"])
    if math.isnan(want):
        assert math.isnan(step[0])
    else:
        assert step[0] == pytest.approx(want, rel=1e-15, abs=1e-12)
    assert hit[0] == case["hit"]


@pytest.mark.parametrize("mode", [0, 1])
def test_edge_cases(g, orc, mode):
    sc = scene("toy40")
    rng = np.random.default_rng(3)
    base = scenes.sample_tracks(sc, 64, 11)
    p = np.stack([base.x, base.y, base.z], 1)
    d = np.stack([base.dx, base.dy, base.dz], 1)
    p[0] = (2000.0, 0, 0)                 # outside the mother
    p[1] = (0, 0, 1500.0)                 # on the mother's top face
    d[2] = 0.0                            # zero direction
    p[3, 0] = np.nan                      # non-finite
    d[4, 1] = np.inf
    p[5] = (0.0, 0.0, 0.0)                # on the axis (inside the innermost hole)
    p[6] = (55.0, 0.0, 0.0)               # inside tube shell 0 (40..70)
    d[7] *= 3.0                           # non-unit direction
    p[8] = (40.0, 0.0, 200.0)             # on the inner wall of shell 0
    p[9] = (750.0, 0.0, 0.0)              # centre of a box daughter
    d[10] = (0.0, 0.0, 1.0)               # along the axis
    p[10] = (300.0, 20.0, -1499.0)
    tr = tracks_from(p, d)
    ref = orc.navigate(sc, tr)
    step, hit = run_nav(g, sc, tr, mode)
    assert hit[0] == -2 and step[0] == 0.0
    assert np.isnan(step[2]) and hit[2] == -2
    assert np.isnan(step[3]) and np.isnan(step[4])
    assert hit[6] == 0 and step[6] == 0.0
    compare(ref, step, hit, tr, sc, orc, max_banded=None)


@pytest.mark.parametrize("n", [0, 1, 31, 255, 257])
def test_small_and_empty_baskets(g, orc, n):
    sc = scene("toy8")
    tr = scenes.sample_tracks(sc, max(n, 1), 12).slice(0, n)
    if n == 0:
        step, hit = run_nav(g, sc, tr, 1)
        assert step.size == 0 and hit.size == 0
        return
    ref = orc.navigate(sc, tr)
    for mode in (0, 1):
        step, hit = run_nav(g, sc, tr, mode)
        compare(ref, step, hit, tr, sc, orc, max_banded=None)


def test_boundary_point(g):
    sc = scene("toy40")
    tr = scenes.sample_tracks(sc, 10000, 13)
    step, hit, bp = run_nav(g, sc, tr, 1, bpoint=True)
    for k, (pc, dc) in enumerate(((tr.x, tr.dx), (tr.y, tr.dy), (tr.z, tr.dz))):
        want = pc + step * dc
        assert np.allclose(bp[k], want, rtol=0, atol=1e-12 * 3000)


@pytest.mark.parametrize("mode", [0, 1])
def test_contains_parity(g, orc, mode):
    for name in SCENES:
        sc = scene(name)
        tr = scenes.sample_tracks(sc, 20000, 14, exclusive=False)
        want = orc.contains(sc, tr, nthreads=8)
        x, y, z = dev(tr)[:3]
        got = g.geo_contains(vol(g, sc), x, y, z, mode=mode).cpu().numpy()
        # surface band: points whose answer changes under a 1e-9 mm move
        band = np.zeros(tr.n, dtype=bool)
        for k in range(3):
            for sg in (-1e-9, 1e-9):
                f = [tr.x.copy(), tr.y.copy(), tr.z.copy()]
                f[k] = f[k] + sg
                band |= orc.contains(sc, scenes.Tracks(*f, tr.dx, tr.dy, tr.dz), nthreads=8) != want
        assert np.array_equal(got[~band], want[~band]), name
        assert band.mean() < 1e-3


@pytest.mark.parametrize("mode", [0, 1])
def test_safety_parity(g, orc, mode):
    for name in SCENES:
        sc = scene(name)
        tr = scenes.sample_tracks(sc, 20000, 15, exclusive=False)
        want = orc.safety(sc, tr, nthreads=8)
        x, y, z = dev(tr)[:3]
        got = g.geo_safety(vol(g, sc), x, y, z, mode=mode).cpu().numpy()
        assert np.max(np.abs(got - want)) <= STEP_TOL, name


@pytest.mark.parametrize("mode,chunk", [(1, 30000), (1, 7001), (0, 50000), (1, 0)])
def test_host_entry_matches_device(g, mode, chunk):
    """The host-buffer pipeline: 4 chunks (one buffer reused), 15 ragged
    chunks (every buffer reused several times), 2 chunks, one chunk."""
    sc = scene("toy40")
    tr = scenes.sample_tracks(sc, 100000, 16)
    s0, h0 = run_nav(g, sc, tr, mode)
    s1, h1 = g.geo_dist_to_boundary_host(vol(g, sc), *tr.fields(), mode=mode, chunk=chunk)
    assert np.array_equal(s0.view(np.int64), s1.view(np.int64))
    assert np.array_equal(h0, h1)


@pytest.mark.parametrize("mode", [0, 1])
def test_host_entry_in_place(g, mode):
    """Pinned host arrays: the step reads and writes them in place (no
    staging); a ragged basket, a small one (the warp-per-track path), and
    pinned inputs with a pageable output (staged again)."""
    import torch

    sc = scene("toy40")
    v = vol(g, sc)
    for n in (100003, 77):
        tr = scenes.sample_tracks(sc, n, 18)
        s0, h0 = run_nav(g, sc, tr, mode)
        pinned = [torch.from_numpy(f).pin_memory() for f in tr.fields()]
        s1, h1 = g.geo_dist_to_boundary_host(v, *pinned, mode=mode)
        assert s1.is_pinned() and h1.is_pinned()
        assert np.array_equal(s0.view(np.int64), s1.numpy().view(np.int64))
        assert np.array_equal(h0, h1.numpy())
        s2, h2 = g.geo_dist_to_boundary_host(v, *pinned, mode=mode, step=np.empty(n),
                                             hit=torch.empty(n, dtype=torch.int32).pin_memory())
        assert np.array_equal(s0.view(np.int64), s2.view(np.int64)) and np.array_equal(h0, h2.numpy())


def test_host_entry_rejects_device_arrays(g):
    import torch

    sc = scene("toy40")
    tr = scenes.sample_tracks(sc, 1000, 19)
    d = [torch.from_numpy(f).cuda() for f in tr.fields()]
    with pytest.raises(g.GeoError):
        g.geo_dist_to_boundary_host(vol(g, sc), *d, mode=1, step=np.empty(1000), hit=np.empty(1000, np.int32))


def test_full_size_toy_detector_sampled(g, orc):
    """The 2^20-track toy-detector basket in the launch configuration the
    benchmark times; the oracle checks a random sample of 20000 tracks."""
    sc = scene("toy40")
    tr = scenes.sample_tracks(sc, 1 << 20, 1)
    step, hit = run_nav(g, sc, tr, 1)
    s64, h64 = run_nav(g, sc, tr, 0)
    assert np.array_equal(step.view(np.int64), s64.view(np.int64)) and np.array_equal(hit, h64)
    idx = np.sort(np.random.default_rng(17).choice(tr.n, 20000, replace=False))
    sub = scenes.Tracks(*(f[idx] for f in tr.fields()))
    ref = orc.navigate(sc, sub, nthreads=8)
    compare(ref, step[idx], hit[idx], sub, sc, orc, max_graze=1e-4)


def many_solids_scene():
    """36 small solids of every kind (boxes, tubes, cones, tube segments,
    polycones), rotated, on a 4 x 3 x 3 grid of pitch 200 mm in a box mother:
    the split kernel's instantiation with the segment and polycone code."""
    rng = np.random.default_rng(41)
    rows = []
    k = 0
    for ix in range(4):
        for iy in range(3):
            for iz in range(3):
                c = (-300.0 + 200.0 * ix, -200.0 + 200.0 * iy, -200.0 + 200.0 * iz)
                rot = scenes.haar_rotation(rng)
                kind = k % 5
                if kind == scenes.BOX:
                    spec = tuple(rng.uniform(15.0, 40.0, 3))
                elif kind == scenes.TUBE:
                    spec = (rng.uniform(0.0, 15.0), rng.uniform(25.0, 45.0), rng.uniform(15.0, 45.0))
                elif kind == scenes.CONE:
                    spec = (rng.uniform(20.0, 40.0), 5.0, 30.0, 0.0, 40.0)
                elif kind == scenes.TUBS:
                    spec = (rng.uniform(0.0, 10.0), rng.uniform(25.0, 45.0), rng.uniform(15.0, 40.0),
                            rng.uniform(-3.0, 3.0), rng.uniform(0.5, 6.0))
                else:
                    spec = scenes.Pcon((-30.0, -5.0, 5.0, 30.0), (0.0, 8.0, 8.0, 0.0), (30.0, 40.0, 40.0, 25.0),
                                       rng.uniform(-3.0, 3.0), rng.uniform(1.0, 2.0 * math.pi))
                rows.append((kind, spec, rot, c))
                k += 1
    return scenes._scene("many36", scenes.BOX, (450.0, 350.0, 350.0), rows)


@pytest.mark.parametrize("name", ["toy40", "grid512", "grid512_vox", "many36"])
def test_split_small_baskets(g, orc, name):
    """Small baskets in volumes of more than 32 daughters take the split
    kernel (a track's FP32 pass spread over the warps of a block by daughter;
    a volume's uniform grid is not walked there): the plain FP64 bits and
    boundary points, the same bits as the pipelined kernel gives the same
    tracks in a large basket, on either side of the switch and on ragged
    block tails; the oracle on the smallest baskets."""
    sc = many_solids_scene() if name == "many36" else scene(name.replace("_vox", ""))
    voxelize = name.endswith("_vox")
    volh = g.geo_build_volume(sc, voxelize=voxelize) if voxelize else vol(g, sc)

    def nav(tr, mode):
        out = g.geo_dist_to_boundary(volh, *dev(tr), mode=mode, want_bpoint=True)
        torch.cuda.synchronize()
        return [o.cpu().numpy() for o in out]

    sms = torch.cuda.get_device_properties(0).multi_processor_count
    edge = 4 * sms * 32 * (2 if sc.n_daughters >= 128 and not voxelize else 1)
    big = scenes.sample_tracks(sc, max(edge + 100, 200000), 51)
    s_big, h_big, b_big = nav(big, 1)
    for n in (1, 31, 33, 1000, edge, edge + 1):
        tr = big.slice(0, n)
        s1, h1, b1 = nav(tr, 1)
        s0, h0, b0 = nav(tr, 0)
        assert np.array_equal(h1, h0) and np.array_equal(s1.view(np.int64), s0.view(np.int64)), (name, n)
        assert np.array_equal(b1.view(np.int64), b0.view(np.int64)), (name, n)
        assert np.array_equal(h1, h_big[:n]) and np.array_equal(s1.view(np.int64), s_big[:n].view(np.int64)), n
        if n <= 1000:
            compare(orc.navigate(sc, tr, nthreads=8), s1, h1, tr, sc, orc, max_banded=None)
    # adversarial rays (grazing, edges, apexes) in a small basket
    adv = scenes.adversarial_tracks(sc, 2000, 52)
    s1, h1, _ = nav(adv, 1)
    s0, h0, _ = nav(adv, 0)
    assert np.array_equal(h1, h0) and np.array_equal(s1.view(np.int64), s0.view(np.int64))
    _, _, nref = g.geo_dist_to_boundary_stats(volh, *dev(big.slice(0, 1000)))
    assert np.all(nref.cpu().numpy() >= 0)
    assert g.geo_check_device_status(volh) == 0
