"""The batched persistent launch (many logical volumes, uneven baskets, one
launch): answers identical to one geo_dist_to_boundary call per basket and to
the oracle; capturable in a CUDA graph."""
import numpy as np
import pytest

from helpers import check_steps
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


@pytest.fixture(scope="module")
def small_batch():
    vols, baskets = scenes.batched64(seed=3, n_volumes=12, total=60000)
    tr, rows = scenes.batched_tracks(vols, baskets, 3)
    return vols, tr, rows


def dev(tr):
    return [torch.from_numpy(np.ascontiguousarray(f)).cuda() for f in tr.fields()]


def per_basket(g, vols, volh, tr, rows, mode):
    step = np.empty(tr.n)
    hit = np.empty(tr.n, dtype=np.int32)
    for v, off, cnt in rows:
        sub = tr.slice(int(off), int(off + cnt))
        s, h = g.geo_dist_to_boundary(volh[int(v)], *dev(sub), mode=mode)
        step[off:off + cnt] = s.cpu().numpy()
        hit[off:off + cnt] = h.cpu().numpy()
    return step, hit


@pytest.mark.parametrize("order,bps,tile", [(0, 0, 0), (1, 0, 0), (0, 1, 0), (0, 0, 256), (1, 1, 256)])
def test_batched_equals_per_basket(g, small_batch, order, bps, tile):
    """Every schedule and both tile shapes (384 tracks, 12 + 4 warps; 256, 8 +
    4) give the per-basket plain FP64 bits."""
    vols, tr, rows = small_batch
    volh = [g.geo_build_volume(v) for v in vols]
    batch = g.geo_build_batch(volh, rows, tile_order=order, blocks_per_sm=bps, tile_tracks=tile)
    s, h = g.geo_dist_to_boundary_batched(batch, *dev(tr))
    torch.cuda.synchronize()
    s, h = s.cpu().numpy(), h.cpu().numpy()
    s64, h64 = per_basket(g, vols, volh, tr, rows, 0)
    assert np.array_equal(h, h64)
    assert np.array_equal(s.view(np.int64), s64.view(np.int64))


def test_batched_oracle_parity(g, orc, small_batch):
    vols, tr, rows = small_batch
    volh = [g.geo_build_volume(v) for v in vols]
    batch = g.geo_build_batch(volh, rows)
    s, h = g.geo_dist_to_boundary_batched(batch, *dev(tr))
    torch.cuda.synchronize()
    s, h = s.cpu().numpy(), h.cpu().numpy()
    for v, off, cnt in rows:
        sub = tr.slice(int(off), int(off + cnt))
        ref = orc.navigate(vols[int(v)], sub, nthreads=8)
        check_steps(ref, s[off:off + cnt], h[off:off + cnt], sub, orc=orc, scene=vols[int(v)])


def test_batched_graph_replay(g, small_batch):
    vols, tr, rows = small_batch
    volh = [g.geo_build_volume(v) for v in vols]
    batch = g.geo_build_batch(volh, rows)
    x = dev(tr)
    step = torch.empty(tr.n, dtype=torch.float64, device="cuda")
    hit = torch.empty(tr.n, dtype=torch.int32, device="cuda")
    g.geo_dist_to_boundary_batched(batch, *x, step=step, hit=hit)   # warm-up outside capture
    torch.cuda.synchronize()
    ref_s, ref_h = step.clone(), hit.clone()
    graph = torch.cuda.CUDAGraph()
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        with torch.cuda.graph(graph, stream=s):
            g.geo_dist_to_boundary_batched(batch, *x, step=step, hit=hit)
    for _ in range(3):
        step.fill_(-1.0)
        hit.fill_(99)
        graph.replay()
        torch.cuda.synchronize()
        assert torch.equal(step, ref_s) and torch.equal(hit, ref_h)


def test_batched_rejects_short_arrays(g, small_batch):
    vols, tr, rows = small_batch
    volh = [g.geo_build_volume(v) for v in vols]
    batch = g.geo_build_batch(volh, rows)
    short = [f[:-1] for f in dev(tr)]
    with pytest.raises(g.GeoError):
        g.geo_dist_to_boundary_batched(batch, *short)


def test_full_batched_workload_sampled(g, orc):
    """64 volumes, ~530 baskets of 16..65536 tracks, 2^22 tracks: one launch,
    bitwise equal to the per-basket FP64 calls on sampled baskets, oracle on a
    sample of tracks."""
    vols, baskets = scenes.batched64(seed=3)
    tr, rows = scenes.batched_tracks(vols, baskets, 3)
    volh = [g.geo_build_volume(v) for v in vols]
    batch = g.geo_build_batch(volh, rows)
    s, h = g.geo_dist_to_boundary_batched(batch, *dev(tr))
    torch.cuda.synchronize()
    s, h = s.cpu().numpy(), h.cpu().numpy()
    rng = np.random.default_rng(1)
    pick = rng.choice(len(rows), 40, replace=False)
    for k in pick:
        v, off, cnt = rows[k]
        sub = tr.slice(int(off), int(off + cnt))
        s64, h64 = g.geo_dist_to_boundary(volh[int(v)], *dev(sub), mode=0)
        assert np.array_equal(h[off:off + cnt], h64.cpu().numpy())
        assert np.array_equal(s[off:off + cnt].view(np.int64), s64.cpu().numpy().view(np.int64))
        n = min(int(cnt), 500)
        ref = orc.navigate(vols[int(v)], sub.slice(0, n), nthreads=8)
        check_steps(ref, s[off:off + n], h[off:off + n], sub.slice(0, n), orc=orc, scene=vols[int(v)])


def test_autotuner_picks_a_candidate_and_caches(g, small_batch, tmp_path, monkeypatch):
    from paper_1312_0816_gb300 import autotune

    monkeypatch.setattr(autotune, "CACHE", str(tmp_path / "tune.json"))
    vols, tr, rows = small_batch
    volh = [g.geo_build_volume(v) for v in vols]
    x = dev(tr)
    step = torch.empty(tr.n, dtype=torch.float64, device="cuda")
    hit = torch.empty(tr.n, dtype=torch.int32, device="cuda")
    order, bps, tile, timings = autotune.tune_batch(volh, rows, x, step, hit, reps=3)
    assert (order, bps, tile) in autotune.CANDIDATES
    assert len(timings) == len(autotune.CANDIDATES) and all(t > 0 for t in timings.values())
    again = autotune.tune_batch(volh, rows, x, step, hit, reps=3)
    assert again[:3] == (order, bps, tile)
    # the tuned schedule gives the same answers
    batch = g.geo_build_batch(volh, rows, tile_order=order, blocks_per_sm=bps, tile_tracks=tile)
    s, h = g.geo_dist_to_boundary_batched(batch, *x)
    ref = g.geo_build_batch(volh, rows)
    s0, h0 = g.geo_dist_to_boundary_batched(ref, *x)
    torch.cuda.synchronize()
    assert torch.equal(s, s0) and torch.equal(h, h0)


def test_batched_segments_and_polycones(g):
    """Volumes with tube segments and polycones (the batched kernel's
    instantiation with their code) mixed with plain ones, baskets of 1 to 700
    tracks (packed ragged tails): the same bits as one call per basket."""
    vols = [scenes.seg4(), scenes.pcon4(), scenes.pconm(), scenes.toy8(1)]
    rng = np.random.default_rng(11)
    baskets = [(int(rng.integers(0, 4)), int(rng.integers(1, 700))) for _ in range(60)]
    tr, rows = scenes.batched_tracks(vols, baskets, 12)
    volh = [g.geo_build_volume(v) for v in vols]
    for order, tile in ((0, 0), (1, 0), (0, 256)):
        batch = g.geo_build_batch(volh, rows, tile_order=order, tile_tracks=tile)
        s, h = g.geo_dist_to_boundary_batched(batch, *dev(tr))
        torch.cuda.synchronize()
        s, h = s.cpu().numpy(), h.cpu().numpy()
        s64, h64 = per_basket(g, vols, volh, tr, rows, 0)
        assert np.array_equal(h, h64)
        assert np.array_equal(s.view(np.int64), s64.view(np.int64))
        batch.close()



@pytest.mark.parametrize("segs", [False, True], ids=["plain", "segments"])
def test_batched_with_voxelised_volumes(g, segs):
    """A batch holding volumes with a uniform grid (the batched kernel's
    instantiation with the grid walk) beside plain ones, with and without
    tube segments and polycones: the same bits as one call per basket, both
    tile shapes."""
    vols = [scenes.grid512(5), scenes.toy40(1), scenes.box4(0)]
    vox = [True, True, False]
    if segs:
        vols.append(scenes.pcon4())
        vox.append(False)
    rng = np.random.default_rng(21)
    baskets = [(int(rng.integers(0, len(vols))), int(rng.integers(1, 900))) for _ in range(50)]
    tr, rows = scenes.batched_tracks(vols, baskets, 13)
    volh = [g.geo_build_volume(v, voxelize=x) for v, x in zip(vols, vox)]
    for tile in (0, 256):
        batch = g.geo_build_batch(volh, rows, tile_order=0, tile_tracks=tile)
        s, h = g.geo_dist_to_boundary_batched(batch, *dev(tr))
        torch.cuda.synchronize()
        s, h = s.cpu().numpy(), h.cpu().numpy()
        s64, h64 = per_basket(g, vols, volh, tr, rows, 0)
        assert np.array_equal(h, h64)
        assert np.array_equal(s.view(np.int64), s64.view(np.int64))
        batch.close()
    for v in volh:
        v.close()
