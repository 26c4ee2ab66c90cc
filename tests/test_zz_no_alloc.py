"""The no-allocation entry point, for callers that cannot let a library
allocate device memory while they run (their allocator owns all device memory,
or allocation is forbidden after start-up).  It must give the same answers as the regular
batched entry point, call after call, while its scratch lives in the
library's fixed device array.  This file is collected last on purpose."""
import numpy as np
import pytest

from paper_1312_0816_gb300 import scenes

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

STEP_TOL = 1e-9   # the parity tolerance of the other GPU tests


def test_noalloc_matches_regular_batched_two_calls():
    import paper_1312_0816_gb300 as g

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    vols, baskets = scenes.batched64(seed=3, n_volumes=12, total=60000)
    tr, rows = scenes.batched_tracks(vols, baskets, 3)
    x = [torch.from_numpy(np.ascontiguousarray(f)).cuda() for f in tr.fields()]
    volh = [g.geo_build_volume(v) for v in vols]
    batch = g.geo_build_batch(volh, rows)
    ref_s, ref_h = g.geo_dist_to_boundary_batched(batch, *x)
    torch.cuda.synchronize()
    ref_s, ref_h = ref_s.cpu().numpy(), ref_h.cpu().numpy()
    step = torch.empty(tr.n, dtype=torch.float64, device="cuda")
    hit = torch.empty(tr.n, dtype=torch.int32, device="cuda")
    for _ in range(2):   # the scratch keeps the previous call's contents
        step.fill_(-1.0)
        hit.fill_(99)
        g.geo_dist_to_boundary_batched_noalloc(volh, rows, *x, step=step, hit=hit)
        torch.cuda.synchronize()
        s, h = step.cpu().numpy(), hit.cpu().numpy()
        assert np.array_equal(h, ref_h)
        assert np.max(np.abs(s - ref_s)) <= STEP_TOL
        assert np.array_equal(s.view(np.int64), ref_s.view(np.int64))


def test_noalloc_rejects_requests_beyond_its_scratch():
    import paper_1312_0816_gb300 as g

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    sc = scenes.box4(0)
    vol = g.geo_build_volume(sc)
    n = 32768 * g.GEO_TILE_TRACKS + 1   # one track more than 32768 full tiles
    x = [torch.zeros(1, dtype=torch.float64, device="cuda").expand(n).contiguous() for _ in range(6)]
    step = torch.empty(n, dtype=torch.float64, device="cuda")
    hit = torch.empty(n, dtype=torch.int32, device="cuda")
    with pytest.raises(g.GeoError):
        g.geo_dist_to_boundary_batched_noalloc([vol], [(0, 0, n)], *x, step=step, hit=hit)
    with pytest.raises(g.GeoError):   # more volumes than the scratch holds
        g.geo_dist_to_boundary_batched_noalloc([vol] * 65, [(0, 0, 1)], *[f[:1] for f in x], step=step[:1],
                                               hit=hit[:1])
