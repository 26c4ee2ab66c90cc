"""The uniform-grid candidate list (voxels): the grid walk only decides which
daughters are examined, so both modes must return exactly the answers of the
plain FP64 loop over all daughters, for any grid."""
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


def dev(tr):
    return [torch.from_numpy(np.ascontiguousarray(f)).cuda() for f in tr.fields()]


def run(g, vol, tr, mode):
    s, h = g.geo_dist_to_boundary(vol, *dev(tr), mode=mode)
    torch.cuda.synchronize()
    return s.cpu().numpy(), h.cpu().numpy()


@pytest.mark.parametrize("name,grid", [("grid512", (0, 0, 0)), ("grid512", (8, 8, 8)), ("grid512", (32, 16, 8)),
                                       ("toy40", (0, 0, 0)), ("diff3", (4, 4, 4)), ("seg4", (4, 4, 4)),
                                       ("pcon4", (4, 4, 4)), ("pconm", (4, 4, 8))])
def test_voxel_modes_equal_plain_loop(g, name, grid):
    sc = scenes.SCENES[name]()
    plain = g.geo_build_volume(sc)
    vox = g.geo_build_volume(sc, voxelize=True, grid=grid)
    info = g.geo_volume_info(vox)
    assert info["voxelized"] and all(k > 0 for k in info["grid"])
    if any(grid):
        assert info["grid"] == tuple(grid)
    for tr in (scenes.sample_tracks(sc, 40000, 7), scenes.adversarial_tracks(sc, 20000, 8)):
        s0, h0 = run(g, plain, tr, 0)
        for mode in (0, 1):
            s, h = run(g, vox, tr, mode)
            assert np.array_equal(h, h0)
            assert np.array_equal(s.view(np.int64), s0.view(np.int64))


def test_voxel_oracle_parity(g, orc):
    sc = scenes.grid512(5)
    vox = g.geo_build_volume(sc, voxelize=True)
    tr = scenes.sample_tracks(sc, 30011, 9)
    ref = orc.navigate(sc, tr, nthreads=8)
    s, h = run(g, vox, tr, 1)
    check_steps(ref, s, h, tr, max_banded=1e-3, orc=orc, scene=sc)


def test_voxel_full_size_sampled(g, orc):
    """2^24 tracks in the 512-daughter volume, the launch the benchmark times;
    the oracle (brute force over all 512 daughters) checks a sample."""
    sc = scenes.grid512(5)
    vox = g.geo_build_volume(sc, voxelize=True)
    tr = scenes.sample_tracks(sc, 1 << 24, 5)
    s, h = run(g, vox, tr, 1)
    idx = np.sort(np.random.default_rng(3).choice(tr.n, 20000, replace=False))
    sub = scenes.Tracks(*(f[idx] for f in tr.fields()))
    ref = orc.navigate(sc, sub, nthreads=8)
    check_steps(ref, s[idx], h[idx], sub, max_banded=1e-3, orc=orc, scene=sc)
