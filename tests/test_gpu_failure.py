"""Failure detection on the GPU without a GPU fault.

* A bounded wait that runs out: geo_selftest_wait_timeout launches one warp
  that waits, with a short poll limit, on a barrier nobody arrives at (the
  failure path of every wait of the pipeline kernels).  The kernel records
  the timeout in the volume's status word and returns; the next
  geo_check_device_status reports GEO_ERR_DEVICE_ASSERT with that bit, and the
  context stays usable: the next step runs and the word reads 0 again.
* Allocation failure: host-side fault injection (geo_debug_fail_alloc) makes
  the k-th allocation of a build fail as out of memory, for every k the build
  makes; the build returns GEO_ERR_OOM (no handle, nothing leaked that a
  later build would trip over) and the same build succeeds once the hook is
  off.
"""
import numpy as np
import pytest

from paper_1312_0816_gb300 import scenes

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

ST_SYNC_TIMEOUT = 4


@pytest.fixture(scope="module")
def g():
    import paper_1312_0816_gb300 as pkg

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    pkg.load()
    return pkg


def test_bounded_wait_runs_out_and_is_reported(g):
    sc = scenes.toy40(1)
    vol = g.geo_build_volume(sc)
    assert g.geo_check_device_status(vol) == 0
    g.geo_selftest_wait_timeout(vol, 256)
    with pytest.raises(g.GeoError) as e:
        g.geo_check_device_status(vol)
    assert e.value.status == 5 and "0x4" in str(e.value)
    # the word was read and cleared; the context still works
    tr = scenes.sample_tracks(sc, 4096, 3)
    x = [torch.from_numpy(f).cuda() for f in tr.fields()]
    s1, h1 = g.geo_dist_to_boundary(vol, *x, mode=1)
    s0, h0 = g.geo_dist_to_boundary(vol, *x, mode=0)
    torch.cuda.synchronize()
    assert torch.equal(s1, s0) and torch.equal(h1, h0)
    assert g.geo_check_device_status(vol) == 0
    vol.close()


def _fails_then_succeeds(g, build, max_allocs=24):
    """build() fails with GEO_ERR_OOM for every injected failure point it
    reaches, and succeeds once the injection point lies past its last
    allocation; returns how many allocations it makes."""
    for k in range(1, max_allocs + 1):
        g.geo_debug_fail_alloc(k)
        try:
            obj = build()
        except g.GeoError as e:
            assert e.status == 3, (k, e)
            continue
        finally:
            g.geo_debug_fail_alloc(0)
        obj.close()
        return k - 1
    raise AssertionError("the build kept failing")


def test_allocation_failures_of_every_build(g):
    sc = scenes.grid512(5)
    n_vol = _fails_then_succeeds(g, lambda: g.geo_build_volume(sc, voxelize=True))
    assert n_vol >= 5                                    # host object, tables, status, voxel lists
    vols, baskets = scenes.batched64(seed=3)
    vols = vols[:4]
    tr, rows = scenes.batched_tracks(vols, [(v, 100 + 50 * v) for v in range(4)], 3)
    volh = [g.geo_build_volume(v) for v in vols]
    n_batch = _fails_then_succeeds(g, lambda: g.geo_build_batch(volh, rows))
    assert n_batch >= 3
    w = scenes.world_toy()
    wv = [g.geo_build_volume(v) for v in w.volumes]
    n_world = _fails_then_succeeds(g, lambda: g.geo_build_world(wv, w.child, w.root))
    assert n_world >= 2
    # after all that, the library still builds and steps normally
    step, hit = g.geo_dist_to_boundary(volh[0], *[torch.from_numpy(f[:100]).cuda() for f in tr.fields()], mode=1)
    torch.cuda.synchronize()
    assert np.all(np.isfinite(step.cpu().numpy()))
    for v in volh + wv:
        v.close()
